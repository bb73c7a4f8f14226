// Plain FP64 CPU oracle for the per-event tree-level squared matrix element
// workflow of arXiv:2106.12631 (RAMBO phase space -> helicity amplitudes ->
// colour sum -> helicity sum).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
// only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
// reference arm load it.  It shares no code, header, table or generator with
// the CUDA path.
//
// What it computes, and where the paper defines it:
//  * RAMBO flat phase space from four uniforms per final-state particle
//    (Sec. 3, "toy" workflow: random numbers -> RAMBO -> matrix elements),
//    following Kleiss, Stirling, Ellis, CPC 40 (1986) 359.
//  * |M|^2 summed over ALL helicities and ALL explicit colours, from Feynman
//    rules (Sec. 2: helicity amplitudes, colour-flow method; Fig. 1 for
//    e+e- -> mu+mu-).  This is the plain definition that the colour-flow /
//    helicity-filtered method reaches exactly: no filtering, no colour
//    decomposition.  Dirac algebra uses explicit 4x4 gamma matrices in the
//    chiral basis; colour uses explicit Gell-Mann matrices T^a = lambda^a / 2
//    and f^abc = -2i Tr([T^a,T^b] T^c).  Diagrams come from a generic
//    recursive tree enumeration over the external legs.
//  * The average over initial spins/colours and the identical-particle
//    factor (Sec. 2, "average of these squared amplitudes").
//  * Forward-mode dual numbers give d(me)/d(random numbers).
//
// Conventions (Peskin & Schroeder): metric (+,-,-,-); quark-gluon vertex
// i g gamma^mu T^a; three-gluon vertex g f^abc [g^{mu nu}(k-p)^rho + ...] with
// all momenta incoming; four-gluon vertex -i g^2 [...]; fermion propagator
// i(p/ + m)/(p^2 - m^2 + i m Gamma); Feynman-gauge gluon/photon propagator
// -i g^{mu nu}/k^2; unitary-gauge Z propagator.
//
// Parity status: every function here is pinned by tests (closed forms for
// e+e- -> mu+mu- and gg -> t tbar, RAMBO invariants and closed-form weights,
// Dirac-spinor identities, SU(3) identities, Ward identity, Lorentz/parity
// invariance, Bose symmetry, finite differences for the dual gradient).

#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <algorithm>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace orc {

// ----------------------------------------------------------------------------
// Scalars: double, and a forward-mode dual number with ND derivative slots.
// ----------------------------------------------------------------------------
constexpr int ND = 16;

struct Dual {
  double v = 0.0;
  double d[ND] = {};
  Dual() = default;
  Dual(double x) : v(x) {}
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v); return r; }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, const Dual& b) { a = a * b; return a; }
inline Dual chain(const Dual& a, double f, double df) { Dual r(f); for (int k = 0; k < ND; ++k) r.d[k] = df * a.d[k]; return r; }
inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
inline Dual log(const Dual& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
inline Dual cos(const Dual& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
inline Dual sin(const Dual& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::sqrt; using std::log; using std::cos; using std::sin;

// Complex numbers over either scalar (std::complex is only defined for
// floating-point types, so the dual path needs its own).
template <class T> struct Cx {
  T re, im;
  Cx() : re(0.0), im(0.0) {}
  Cx(const T& r) : re(r), im(0.0) {}
  Cx(const T& r, const T& i) : re(r), im(i) {}
};
template <class T> Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) { return {a.re + b.re, a.im + b.im}; }
template <class T> Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) { return {a.re - b.re, a.im - b.im}; }
template <class T> Cx<T> operator-(const Cx<T>& a) { return {-a.re, -a.im}; }
template <class T> Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
template <class T> Cx<T> operator*(const Cx<T>& a, const T& s) { return {a.re * s, a.im * s}; }
template <class T> Cx<T> operator*(const T& s, const Cx<T>& a) { return {a.re * s, a.im * s}; }
template <class T> Cx<T> conj(const Cx<T>& a) { return {a.re, -a.im}; }
template <class T> T norm2(const Cx<T>& a) { return a.re * a.re + a.im * a.im; }
template <class T> Cx<T> operator/(const Cx<T>& a, const Cx<T>& b) {
  T den = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
template <class T> Cx<T>& operator+=(Cx<T>& a, const Cx<T>& b) { a = a + b; return a; }
// constant complex (double) times complex<T>
template <class T> Cx<T> cmul(std::complex<double> c, const Cx<T>& a) {
  return {a.re * T(c.real()) - a.im * T(c.imag()), a.re * T(c.imag()) + a.im * T(c.real())};
}

template <class T> using Vec4 = std::array<Cx<T>, 4>;  // Lorentz vector (upper index) or Dirac spinor
template <class T> using Mom = std::array<T, 4>;       // real four-momentum (E, px, py, pz)
using CMat4 = std::array<std::array<std::complex<double>, 4>, 4>;

// ----------------------------------------------------------------------------
// Dirac matrices, chiral (Weyl) basis:  gamma^0 = [[0,1],[1,0]],
// gamma^k = [[0, sigma^k], [-sigma^k, 0]], gamma5 = diag(-1,-1,1,1); the upper
// two components are left-handed (the HELAS convention that the paper's
// wavefunctions follow, Sec. 2).
// ----------------------------------------------------------------------------
struct Dirac {
  CMat4 g[4];
  CMat4 g5;
  Dirac() {
    using C = std::complex<double>;
    const C I(0, 1);
    C sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    for (auto& m : g) for (auto& r : m) r.fill(0);
    for (auto& r : g5) r.fill(0);
    for (int a = 0; a < 2; ++a) { g[0][a][a + 2] = 1; g[0][a + 2][a] = 1; }
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) { g[k + 1][a][b + 2] = sig[k][a][b]; g[k + 1][a + 2][b] = -sig[k][a][b]; }
    g5[0][0] = -1; g5[1][1] = -1; g5[2][2] = 1; g5[3][3] = 1;
  }
};
static const Dirac& dirac() { static Dirac d; return d; }

static const double kMetric[4] = {1.0, -1.0, -1.0, -1.0};

template <class T> T mdot(const Mom<T>& a, const Mom<T>& b) { return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]; }
template <class T> Cx<T> cdot(const Vec4<T>& a, const Vec4<T>& b) {  // a^mu b_mu, no conjugation
  Cx<T> r = a[0] * b[0];
  r = r - a[1] * b[1]; r = r - a[2] * b[2]; r = r - a[3] * b[3];
  return r;
}
template <class T> Vec4<T> mom_to_vec(const Mom<T>& p) { return {Cx<T>(p[0]), Cx<T>(p[1]), Cx<T>(p[2]), Cx<T>(p[3])}; }

// slash(A) = gamma^mu A_mu  (4x4 matrix with entries Cx<T>)
template <class T> using Mat4 = std::array<std::array<Cx<T>, 4>, 4>;
template <class T> Mat4<T> slash(const Vec4<T>& A) {
  const Dirac& D = dirac();
  Mat4<T> M;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      Cx<T> s;
      for (int mu = 0; mu < 4; ++mu) s += cmul(D.g[mu][i][j] * kMetric[mu], A[mu]);
      M[i][j] = s;
    }
  return M;
}
template <class T> Vec4<T> mat_col(const Mat4<T>& M, const Vec4<T>& c) {
  Vec4<T> r;
  for (int i = 0; i < 4; ++i) { Cx<T> s; for (int j = 0; j < 4; ++j) s += M[i][j] * c[j]; r[i] = s; }
  return r;
}
template <class T> Vec4<T> row_mat(const Vec4<T>& w, const Mat4<T>& M) {
  Vec4<T> r;
  for (int j = 0; j < 4; ++j) { Cx<T> s; for (int i = 0; i < 4; ++i) s += w[i] * M[i][j]; r[j] = s; }
  return r;
}
template <class T> Vec4<T> cmat_col(const CMat4& M, const Vec4<T>& c) {
  Vec4<T> r;
  for (int i = 0; i < 4; ++i) { Cx<T> s; for (int j = 0; j < 4; ++j) s += cmul(M[i][j], c[j]); r[i] = s; }
  return r;
}
template <class T> Cx<T> row_col(const Vec4<T>& w, const Vec4<T>& c) {
  Cx<T> s; for (int i = 0; i < 4; ++i) s += w[i] * c[i]; return s;
}
// row . gamma^mu . col for mu = 0..3 (upper index)
template <class T> Vec4<T> bilinear(const Vec4<T>& row, const Vec4<T>& col) {
  const Dirac& D = dirac();
  Vec4<T> r;
  for (int mu = 0; mu < 4; ++mu) r[mu] = row_col(row, cmat_col(D.g[mu], col));
  return r;
}
// chirality projectors applied to a column: gL PL + gR PR with PL = diag(1,1,0,0)
template <class T> Vec4<T> chiral_col(const Vec4<T>& c, double gl, double gr) {
  return {c[0] * T(gl), c[1] * T(gl), c[2] * T(gr), c[3] * T(gr)};
}
template <class T> Vec4<T> scale(const Vec4<T>& a, const Cx<T>& s) { return {a[0] * s, a[1] * s, a[2] * s, a[3] * s}; }
template <class T> Vec4<T> add(const Vec4<T>& a, const Vec4<T>& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2], a[3] + b[3]}; }
template <class T> Vec4<T> sub(const Vec4<T>& a, const Vec4<T>& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2], a[3] - b[3]}; }
// Dirac adjoint of a column spinor: psi^dagger gamma^0
template <class T> Vec4<T> dirac_bar(const Vec4<T>& c) {
  Vec4<T> cc = {conj(c[0]), conj(c[1]), conj(c[2]), conj(c[3])};
  // gamma^0 swaps the upper and lower pairs
  return {cc[2], cc[3], cc[0], cc[1]};
}

// ----------------------------------------------------------------------------
// External wavefunctions (Sec. 2: "external particle" routines, IXXXXX for
// the flowing-in and OXXXXX for the flowing-out fermions; vector bosons).
// Helicity eigenspinors chi_lambda(p^) of sigma.p^ with eigenvalue lambda.
// ----------------------------------------------------------------------------
template <class T> void helicity_chi(const Mom<T>& p, int lam, Cx<T> chi[2]) {
  T pt2 = p[1] * p[1] + p[2] * p[2];
  T pp = sqrt(pt2 + p[3] * p[3]);
  // |p| + pz, written as pT^2 / (|p| - pz) for pz < 0 (the same number without
  // cancellation for momenta close to -z)
  T ppz = val(p[3]) >= 0 ? pp + p[3] : pt2 / (pp - p[3]);
  if (val(ppz) <= 0.0) {  // momentum exactly along -z: fixed phase choice
    if (lam > 0) { chi[0] = Cx<T>(T(0.0)); chi[1] = Cx<T>(T(1.0)); }
    else { chi[0] = Cx<T>(T(-1.0)); chi[1] = Cx<T>(T(0.0)); }
    return;
  }
  T nrm = T(1.0) / sqrt(T(2.0) * pp * ppz);
  if (lam > 0) { chi[0] = Cx<T>(ppz * nrm); chi[1] = Cx<T>(p[1] * nrm, p[2] * nrm); }
  else { chi[0] = Cx<T>(-p[1] * nrm, p[2] * nrm); chi[1] = Cx<T>(ppz * nrm); }
}
// omega_{+-} = sqrt(E +- |p|); massless: omega_- is exactly zero
template <class T> void omegas(const Mom<T>& p, double m, T& wp, T& wm) {
  T pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  wp = sqrt(p[0] + pp);
  if (m == 0.0) wm = T(0.0);
  else wm = T(m) / wp;  // sqrt(E-|p|) = m / sqrt(E+|p|), free of cancellation
}
// u(p, lam) = ( omega_{-lam} chi_lam , omega_{+lam} chi_lam )
template <class T> Vec4<T> spinor_u(const Mom<T>& p, double m, int lam) {
  Cx<T> chi[2]; helicity_chi(p, lam, chi);
  T wp, wm; omegas(p, m, wp, wm);
  T lo = lam > 0 ? wm : wp, hi = lam > 0 ? wp : wm;
  return {chi[0] * lo, chi[1] * lo, chi[0] * hi, chi[1] * hi};
}
// v(p, lam) = ( -lam omega_{lam} chi_{-lam} , lam omega_{-lam} chi_{-lam} )
template <class T> Vec4<T> spinor_v(const Mom<T>& p, double m, int lam) {
  Cx<T> chi[2]; helicity_chi(p, -lam, chi);
  T wp, wm; omegas(p, m, wp, wm);
  T wl = lam > 0 ? wp : wm, wml = lam > 0 ? wm : wp;
  T a = T(-double(lam)) * wl, b = T(double(lam)) * wml;
  return {chi[0] * a, chi[1] * a, chi[0] * b, chi[1] * b};
}
// massless vector polarisation eps(k, lam) = (-lam e1 - i e2)/sqrt2
template <class T> Vec4<T> polvec(const Mom<T>& k, int lam) {
  T kt = sqrt(k[1] * k[1] + k[2] * k[2]);
  T kk = sqrt(kt * kt + k[3] * k[3]);
  T ct, st, cp, sp;
  if (val(kt) <= 1e-14 * val(kk)) {
    ct = T(val(k[3]) > 0 ? 1.0 : -1.0); st = T(0.0); cp = T(1.0); sp = T(0.0);
  } else {
    ct = k[3] / kk; st = kt / kk; cp = k[1] / kt; sp = k[2] / kt;
  }
  const double r2 = 1.0 / std::sqrt(2.0);
  T e1[4] = {T(0.0), ct * cp, ct * sp, -st};
  T e2[4] = {T(0.0), -sp, cp, T(0.0)};
  Vec4<T> e;
  for (int mu = 0; mu < 4; ++mu) e[mu] = Cx<T>(T(-double(lam) * r2) * e1[mu], T(-r2) * e2[mu]);
  return e;
}

// ----------------------------------------------------------------------------
// SU(3) colour: Gell-Mann generators and structure constants.
// ----------------------------------------------------------------------------
using C = std::complex<double>;
struct SU3 {
  C T[8][3][3];
  double f[8][8][8];
  SU3() {
    const C I(0, 1);
    C lam[8][3][3] = {};
    lam[0][0][1] = 1; lam[0][1][0] = 1;
    lam[1][0][1] = -I; lam[1][1][0] = I;
    lam[2][0][0] = 1; lam[2][1][1] = -1;
    lam[3][0][2] = 1; lam[3][2][0] = 1;
    lam[4][0][2] = -I; lam[4][2][0] = I;
    lam[5][1][2] = 1; lam[5][2][1] = 1;
    lam[6][1][2] = -I; lam[6][2][1] = I;
    const double s3 = 1.0 / std::sqrt(3.0);
    lam[7][0][0] = s3; lam[7][1][1] = s3; lam[7][2][2] = -2.0 * s3;
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[a][i][j] = 0.5 * lam[a][i][j];
    // f^abc = -2 i Tr([T^a, T^b] T^c)
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        for (int c = 0; c < 8; ++c) {
          C tr = 0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              for (int k = 0; k < 3; ++k)
                tr += (T[a][i][j] * T[b][j][k] - T[b][i][j] * T[a][j][k]) * T[c][k][i];
          C v = C(0, -2) * tr;
          f[a][b][c] = std::abs(v.real()) < 1e-14 ? 0.0 : v.real();
        }
  }
};
static const SU3& su3() { static SU3 s; return s; }

// ----------------------------------------------------------------------------
// Processes.  Every external leg is described by its line type as seen from
// the diagram when all momenta are taken outgoing (crossing): a "row" fermion
// ends the fermion line (u-bar or v-bar), a "col" fermion starts it (u or v).
// ----------------------------------------------------------------------------
enum Line { GLU = 0, PHO, ZB, ROW_T, COL_T, ROW_E, COL_E, ROW_M, COL_M, NLINE };
static bool is_row(Line l) { return l == ROW_T || l == ROW_E || l == ROW_M; }
static bool is_col(Line l) { return l == COL_T || l == COL_E || l == COL_M; }
static int flavour(Line l) { return (l == ROW_T || l == COL_T) ? 0 : (l == ROW_E || l == COL_E) ? 1 : 2; }
static Line row_of(int fl) { return fl == 0 ? ROW_T : fl == 1 ? ROW_E : ROW_M; }
static Line col_of(int fl) { return fl == 0 ? COL_T : fl == 1 ? COL_E : COL_M; }
static bool is_vec(Line l) { return l == GLU || l == PHO || l == ZB; }
static int colour_dim(Line l) { return l == GLU ? 8 : (l == ROW_T || l == COL_T) ? 3 : 1; }

struct Leg {
  Line line;
  bool incoming;
  bool particle;  // fermion: particle (u / u-bar) or antiparticle (v / v-bar)
  int mass_id;    // 0 massless, 1 top
};
struct Process {
  int id;
  std::vector<Leg> legs;
  double hel_avg, col_avg, sym;
};
static Process make_process(int id) {
  Process P;
  P.id = id;
  P.hel_avg = 4.0;
  switch (id) {
    case 1:  // e+ e- -> mu+ mu-
      P.legs = {{ROW_E, true, false, 0}, {COL_E, true, true, 0}, {COL_M, false, false, 0}, {ROW_M, false, true, 0}};
      P.col_avg = 1.0; P.sym = 1.0; break;
    case 2:  // g g -> t t~
      P.legs = {{GLU, true, true, 0}, {GLU, true, true, 0}, {ROW_T, false, true, 1}, {COL_T, false, false, 1}};
      P.col_avg = 64.0; P.sym = 1.0; break;
    case 3:  // g g -> t t~ g
      P.legs = {{GLU, true, true, 0}, {GLU, true, true, 0}, {ROW_T, false, true, 1}, {COL_T, false, false, 1}, {GLU, false, true, 0}};
      P.col_avg = 64.0; P.sym = 1.0; break;
    case 4:  // g g -> t t~ g g
      P.legs = {{GLU, true, true, 0}, {GLU, true, true, 0}, {ROW_T, false, true, 1}, {COL_T, false, false, 1}, {GLU, false, true, 0}, {GLU, false, true, 0}};
      P.col_avg = 64.0; P.sym = 2.0; break;
    default: P.legs.clear();
  }
  return P;
}

// ----------------------------------------------------------------------------
// Tree-diagram enumeration.  The last leg is the root; every other leg set S
// gets the list of all off-shell sub-trees ("nodes") whose external legs are
// exactly S.  A node is a vertex joining 2 (or, for the four-gluon vertex, 3)
// child nodes whose leg sets partition S; each unordered partition is taken
// once.  The four-gluon vertex is split into its three colour/Lorentz terms,
// so every node carries one colour tensor and one kinematic factor.
// ----------------------------------------------------------------------------
enum VKind { V_EXT, V_QQG_ROW, V_QQG_COL, V_QQG_PAIR, V_GGG, V_GGGG, V_FFA_ROW, V_FFA_COL, V_FFA_PAIR, V_FFZ_ROW, V_FFZ_COL, V_FFZ_PAIR };
struct Node {
  VKind kind;
  int term = 0;          // four-gluon term 0..2
  uint32_t mask = 0;     // external legs below this node
  Line out;              // line type leaving the node towards the root
  int child[3] = {-1, -1, -1};
  int nchild = 0;
  int leg = -1;          // for V_EXT
  int n4g = 0;           // number of four-gluon vertices in the sub-tree
  int t4g_nonzero = 0;   // number of four-gluon vertices with term != 0
};

struct Topology {
  Process proc;
  std::vector<Node> nodes;
  std::map<uint32_t, std::vector<int>> by_mask;
  std::vector<int> amps;        // nodes (leg set = all but the root) closing on the root
  int ndiagrams = 0;            // four-gluon vertex counted once
  // colour
  std::vector<std::vector<C>> ctensor;  // per node: [legs in mask order][open]
  std::vector<std::vector<C>> cc;       // per amplitude pair: sum over colours c_d conj(c_d')
};

static void combine_rules(Line a, Line b, std::vector<std::pair<Line, VKind>>& out) {
  // a, b are the child lines in the order given; rules are looked up in both orders by the caller
  if (a == GLU && b == GLU) out.push_back({GLU, V_GGG});
  if (is_row(a) && b == GLU && flavour(a) == 0) out.push_back({a, V_QQG_ROW});
  if (is_col(a) && b == GLU && flavour(a) == 0) out.push_back({a, V_QQG_COL});
  if (is_row(a) && is_col(b) && flavour(a) == flavour(b)) {
    if (flavour(a) == 0) out.push_back({GLU, V_QQG_PAIR});
    else { out.push_back({PHO, V_FFA_PAIR}); out.push_back({ZB, V_FFZ_PAIR}); }
  }
  if (is_row(a) && flavour(a) != 0 && b == PHO) out.push_back({a, V_FFA_ROW});
  if (is_col(a) && flavour(a) != 0 && b == PHO) out.push_back({a, V_FFA_COL});
  if (is_row(a) && flavour(a) != 0 && b == ZB) out.push_back({a, V_FFZ_ROW});
  if (is_col(a) && flavour(a) != 0 && b == ZB) out.push_back({a, V_FFZ_COL});
}

static Line root_partner(Line root) {
  if (is_row(root)) return col_of(flavour(root));
  if (is_col(root)) return row_of(flavour(root));
  return root;  // vectors close on the same vector type
}

static void build_nodes(Topology& tp, uint32_t S) {
  if (tp.by_mask.count(S)) return;
  if (__builtin_popcount(S) == 1) {
    int leg = __builtin_ctz(S);
    Node n; n.kind = V_EXT; n.mask = S; n.out = tp.proc.legs[leg].line; n.leg = leg;
    tp.nodes.push_back(n);
    tp.by_mask[S].push_back((int)tp.nodes.size() - 1);
    return;
  }
  const uint32_t low = S & (~S + 1u);
  std::vector<int> made;
  // two-part partitions {S1, S2}, S1 holding the lowest leg
  for (uint32_t S1 = (S - 1) & S; S1; S1 = (S1 - 1) & S) {
    if (!(S1 & low)) continue;
    uint32_t S2 = S & ~S1;
    build_nodes(tp, S1); build_nodes(tp, S2);
    std::vector<int> n1 = tp.by_mask[S1], n2 = tp.by_mask[S2];
    for (int i1 : n1)
      for (int i2 : n2) {
        for (int order = 0; order < 2; ++order) {
          int ca = order == 0 ? i1 : i2, cb = order == 0 ? i2 : i1;
          Line la = tp.nodes[ca].out, lb = tp.nodes[cb].out;
          if (order == 1 && la == lb) continue;  // symmetric pair already tried
          std::vector<std::pair<Line, VKind>> rules;
          combine_rules(la, lb, rules);
          for (auto& r : rules) {
            Node n; n.kind = r.second; n.mask = S; n.out = r.first;
            n.child[0] = ca; n.child[1] = cb; n.nchild = 2;
            n.n4g = tp.nodes[ca].n4g + tp.nodes[cb].n4g;
            n.t4g_nonzero = tp.nodes[ca].t4g_nonzero + tp.nodes[cb].t4g_nonzero;
            made.push_back((int)tp.nodes.size());
            tp.nodes.push_back(n);
          }
        }
      }
  }
  // three-part partitions for the four-gluon vertex
  for (uint32_t S1 = (S - 1) & S; S1; S1 = (S1 - 1) & S) {
    if (!(S1 & low)) continue;
    uint32_t R = S & ~S1;
    const uint32_t low2 = R & (~R + 1u);
    for (uint32_t S2 = (R - 1) & R; S2; S2 = (S2 - 1) & R) {
      if (!(S2 & low2)) continue;
      uint32_t S3 = R & ~S2;
      build_nodes(tp, S1); build_nodes(tp, S2); build_nodes(tp, S3);
      for (int i1 : tp.by_mask[S1])
        for (int i2 : tp.by_mask[S2])
          for (int i3 : tp.by_mask[S3]) {
            if (tp.nodes[i1].out != GLU || tp.nodes[i2].out != GLU || tp.nodes[i3].out != GLU) continue;
            for (int t = 0; t < 3; ++t) {
              Node n; n.kind = V_GGGG; n.term = t; n.mask = S; n.out = GLU;
              n.child[0] = i1; n.child[1] = i2; n.child[2] = i3; n.nchild = 3;
              n.n4g = 1 + tp.nodes[i1].n4g + tp.nodes[i2].n4g + tp.nodes[i3].n4g;
              n.t4g_nonzero = (t != 0) + tp.nodes[i1].t4g_nonzero + tp.nodes[i2].t4g_nonzero + tp.nodes[i3].t4g_nonzero;
              made.push_back((int)tp.nodes.size());
              tp.nodes.push_back(n);
            }
          }
    }
  }
  tp.by_mask[S] = made;
}

// colour tensor of a node over the colour indices of its legs (increasing leg
// order) and its open index
static void node_colour(Topology& tp, int id) {
  const Node& n = tp.nodes[id];
  const auto& legs = tp.proc.legs;
  const SU3& G = su3();
  std::vector<int> mlegs;
  for (int l = 0; l < (int)legs.size(); ++l) if (n.mask >> l & 1u) mlegs.push_back(l);
  auto dimof = [&](int l) { return colour_dim(legs[l].line); };
  int odim = colour_dim(n.out);
  size_t nass = 1; for (int l : mlegs) nass *= dimof(l);
  std::vector<C> t(nass * odim, C(0));
  if (n.kind == V_EXT) {
    for (int c = 0; c < odim; ++c) t[c * odim + c] = 1.0;
    tp.ctensor[id] = t; return;
  }
  // for each child: the list of its legs and the open dimension
  int nc = n.nchild;
  std::vector<int> clegs[3];
  int cod[3];
  for (int k = 0; k < nc; ++k) {
    const Node& ch = tp.nodes[n.child[k]];
    for (int l = 0; l < (int)legs.size(); ++l) if (ch.mask >> l & 1u) clegs[k].push_back(l);
    cod[k] = colour_dim(ch.out);
  }
  // vertex colour tensor V[x][y][(z)][o] as a sparse list
  struct Ent { int x, y, z, o; C v; };
  std::vector<Ent> ents;
  switch (n.kind) {
    case V_QQG_ROW:  // (row i, glu a) -> row j : T^a_ij
      for (int i = 0; i < 3; ++i) for (int a = 0; a < 8; ++a) for (int j = 0; j < 3; ++j)
        if (G.T[a][i][j] != C(0)) ents.push_back({i, a, 0, j, G.T[a][i][j]});
      break;
    case V_QQG_COL:  // (col j, glu a) -> col i : T^a_ij
      for (int j = 0; j < 3; ++j) for (int a = 0; a < 8; ++a) for (int i = 0; i < 3; ++i)
        if (G.T[a][i][j] != C(0)) ents.push_back({j, a, 0, i, G.T[a][i][j]});
      break;
    case V_QQG_PAIR:  // (row i, col j) -> glu a : T^a_ij
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int a = 0; a < 8; ++a)
        if (G.T[a][i][j] != C(0)) ents.push_back({i, j, 0, a, G.T[a][i][j]});
      break;
    case V_GGG:
      for (int a = 0; a < 8; ++a) for (int b = 0; b < 8; ++b) for (int c = 0; c < 8; ++c)
        if (G.f[a][b][c] != 0) ents.push_back({a, b, 0, c, C(G.f[a][b][c])});
      break;
    case V_GGGG:
      for (int a = 0; a < 8; ++a) for (int b = 0; b < 8; ++b) for (int c = 0; c < 8; ++c) for (int d = 0; d < 8; ++d) {
        double s = 0;
        for (int e = 0; e < 8; ++e) {
          if (n.term == 0) s += G.f[a][b][e] * G.f[c][d][e];
          else if (n.term == 1) s += G.f[a][c][e] * G.f[b][d][e];
          else s += G.f[a][d][e] * G.f[b][c][e];
        }
        if (std::abs(s) > 1e-15) ents.push_back({a, b, c, d, C(s)});
      }
      break;
    default:  // colourless lepton vertices
      ents.push_back({0, 0, 0, 0, C(1)});
  }
  const std::vector<C>* ct[3];
  for (int k = 0; k < nc; ++k) ct[k] = &tp.ctensor[n.child[k]];
  // enumerate colour assignments of this node's legs
  std::vector<int> cidx(mlegs.size(), 0);
  for (size_t A = 0; A < nass; ++A) {
    size_t rem = A;
    for (int p = (int)mlegs.size() - 1; p >= 0; --p) { cidx[p] = (int)(rem % dimof(mlegs[p])); rem /= dimof(mlegs[p]); }
    size_t base[3];
    for (int k = 0; k < nc; ++k) {
      size_t b = 0;
      for (int l : clegs[k]) {
        int pos = 0; while (mlegs[pos] != l) ++pos;
        b = b * dimof(l) + cidx[pos];
      }
      base[k] = b * cod[k];
    }
    for (const Ent& e : ents) {
      C v = e.v * (*ct[0])[base[0] + e.x] * (*ct[1])[base[1] + e.y];
      if (nc == 3) v *= (*ct[2])[base[2] + e.z];
      if (v != C(0)) t[A * odim + e.o] += v;
    }
  }
  tp.ctensor[id] = t;
}

static Topology* build_topology(int proc) {
  Topology* tp = new Topology();
  tp->proc = make_process(proc);
  int n = (int)tp->proc.legs.size();
  if (n == 0) { delete tp; return nullptr; }
  uint32_t rest = (1u << (n - 1)) - 1u;
  build_nodes(*tp, rest);
  Line want = root_partner(tp->proc.legs[n - 1].line);
  for (int id : tp->by_mask[rest]) {
    // a leg set equal to all-but-root with a single external leg cannot close (n >= 4)
    if (tp->nodes[id].out == want && tp->nodes[id].kind != V_EXT) {
      tp->amps.push_back(id);
      if (tp->nodes[id].t4g_nonzero == 0) tp->ndiagrams++;
    }
  }
  tp->ctensor.resize(tp->nodes.size());
  for (size_t i = 0; i < tp->nodes.size(); ++i) node_colour(*tp, (int)i);  // children precede parents
  // amplitude colour tensors: the open index of the rest node is the root leg's colour,
  // which is the last index in leg order
  size_t na = tp->amps.size();
  tp->cc.assign(na, std::vector<C>(na, C(0)));
  for (size_t d = 0; d < na; ++d)
    for (size_t e = d; e < na; ++e) {
      const auto& x = tp->ctensor[tp->amps[d]];
      const auto& y = tp->ctensor[tp->amps[e]];
      C s = 0;
      for (size_t k = 0; k < x.size(); ++k) if (x[k] != C(0) && y[k] != C(0)) s += x[k] * std::conj(y[k]);
      tp->cc[d][e] = s;
      tp->cc[e][d] = std::conj(s);
    }
  return tp;
}

static Topology* topology(int proc) {
  static std::mutex mu;
  static Topology* cache[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  if (proc < 1 || proc > 4) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!cache[proc]) cache[proc] = build_topology(proc);
  return cache[proc];
}

}  // namespace orc

// ----------------------------------------------------------------------------
// Parameters (Standard-Model inputs of the four processes)
// ----------------------------------------------------------------------------
extern "C" {
typedef struct {
  double mz, wz;       // Z mass and width [GeV]
  double alpha_inv;    // 1/alpha_em
  double sw2;          // sin^2 theta_W
  double mt, wt;       // top mass and width [GeV]
  double alpha_s;      // strong coupling
} oracle_params;
}

namespace orc {

struct Couplings {
  double e, gz, glz, grz, gs;  // e, e/(sw cw), Z couplings of charged leptons, g_s
  double mz, wz, mt, wt;
  double mass(int id) const { return id == 1 ? mt : 0.0; }
  double width(Line l) const { return (l == ROW_T || l == COL_T) ? wt : 0.0; }
  double fmass(Line l) const { return (l == ROW_T || l == COL_T) ? mt : 0.0; }
};
static Couplings couplings(const oracle_params& p) {
  Couplings c;
  c.e = std::sqrt(4.0 * M_PI / p.alpha_inv);
  double cw2 = 1.0 - p.sw2;
  c.gz = c.e / std::sqrt(p.sw2 * cw2);
  c.glz = -0.5 + p.sw2;  // T3 - Q sw2 with Q = -1, T3 = -1/2
  c.grz = p.sw2;         // -Q sw2
  c.gs = std::sqrt(4.0 * M_PI * p.alpha_s);
  c.mz = p.mz; c.wz = p.wz; c.mt = p.mt; c.wt = p.wt;
  return c;
}

// ----------------------------------------------------------------------------
// Kinematic evaluation of every node for one helicity assignment.
// ----------------------------------------------------------------------------
template <class T>
struct Eval {
  const Topology& tp;
  const Couplings& cp;
  std::vector<Mom<T>> kout;      // all-outgoing momentum of each leg
  std::vector<Vec4<T>> amput;    // amputated value of each node
  std::vector<Vec4<T>> cur;      // value with propagator (current)
  std::vector<Mom<T>> K;         // outgoing momentum sum of each node
  int ov_leg = -1;               // optional replacement of one external wavefunction
  Vec4<T> ov_val;
  Eval(const Topology& t, const Couplings& c) : tp(t), cp(c) {}

  Vec4<T> external(int leg, const Mom<T>& p, int lam) {
    if (leg == ov_leg) return ov_val;
    const Leg& L = tp.proc.legs[leg];
    double m = cp.mass(L.mass_id);
    if (L.line == GLU) {
      Vec4<T> e = polvec(p, lam);
      if (!L.incoming) for (auto& x : e) x = conj(x);
      return e;
    }
    if (is_col(L.line)) return L.particle ? spinor_u(p, m, lam) : spinor_v(p, m, lam);
    // row: u-bar (outgoing particle) or v-bar (incoming antiparticle)
    return dirac_bar(L.particle ? spinor_u(p, m, lam) : spinor_v(p, m, lam));
  }

  void run(const std::vector<Mom<T>>& p, const std::vector<int>& hel) {
    size_t nn = tp.nodes.size();
    amput.assign(nn, Vec4<T>());
    cur.assign(nn, Vec4<T>());
    K.assign(nn, Mom<T>());
    const Cx<T> I(T(0.0), T(1.0));
    const T gs(cp.gs), e(cp.e), gz(cp.gz);
    for (size_t id = 0; id < nn; ++id) {
      const Node& n = tp.nodes[id];
      Vec4<T> out;
      if (n.kind == V_EXT) {
        const Leg& L = tp.proc.legs[n.leg];
        Mom<T> k = p[n.leg];
        if (L.incoming) for (auto& x : k) x = -x;
        K[id] = k;
        cur[id] = amput[id] = external(n.leg, p[n.leg], hel[n.leg]);
        continue;
      }
      Mom<T> Ks;
      for (int mu = 0; mu < 4; ++mu) { Ks[mu] = T(0.0); for (int c = 0; c < n.nchild; ++c) Ks[mu] += K[n.child[c]][mu]; }
      K[id] = Ks;
      const Vec4<T>& A = cur[n.child[0]];
      const Vec4<T>& B = cur[n.child[1]];
      switch (n.kind) {
        case V_QQG_ROW: out = row_mat(A, slash(scale(B, I * gs))); break;
        case V_QQG_COL: out = mat_col(slash(scale(B, I * gs)), A); break;
        case V_QQG_PAIR: out = scale(bilinear(A, B), I * gs); break;
        case V_FFA_ROW: out = row_mat(A, slash(scale(B, I * e))); break;  // -i e Q, Q = -1
        case V_FFA_COL: out = mat_col(slash(scale(B, I * e)), A); break;
        case V_FFA_PAIR: out = scale(bilinear(A, B), I * e); break;
        case V_FFZ_ROW: {
          Vec4<T> r = row_mat(A, slash(scale(B, -I * gz)));
          out = {r[0] * T(cp.glz), r[1] * T(cp.glz), r[2] * T(cp.grz), r[3] * T(cp.grz)};  // row . PL/PR
          break;
        }
        case V_FFZ_COL: out = mat_col(slash(scale(B, -I * gz)), chiral_col(A, cp.glz, cp.grz)); break;
        case V_FFZ_PAIR: out = scale(bilinear(A, chiral_col(B, cp.glz, cp.grz)), -I * gz); break;
        case V_GGG: {
          // legs (A, q1 = -K1), (B, q2 = -K2), (out, q3 = K1 + K2); all incoming
          Mom<T> q1, q2, q3;
          for (int mu = 0; mu < 4; ++mu) { q1[mu] = -K[n.child[0]][mu]; q2[mu] = -K[n.child[1]][mu]; q3[mu] = Ks[mu]; }
          Mom<T> d12, d23, d31;
          for (int mu = 0; mu < 4; ++mu) { d12[mu] = q1[mu] - q2[mu]; d23[mu] = q2[mu] - q3[mu]; d31[mu] = q3[mu] - q1[mu]; }
          Cx<T> AB = cdot(A, B), dA = cdot(mom_to_vec(d23), A), dB = cdot(mom_to_vec(d31), B);
          for (int mu = 0; mu < 4; ++mu) out[mu] = (AB * d12[mu] + B[mu] * dA + A[mu] * dB) * gs;
          break;
        }
        case V_GGGG: {
          const Vec4<T>& Cc = cur[n.child[2]];
          Cx<T> AB = cdot(A, B), AC = cdot(A, Cc), BC = cdot(B, Cc);
          Vec4<T> L;
          if (n.term == 0) L = sub(scale(B, AC), scale(A, BC));
          else if (n.term == 1) L = sub(scale(Cc, AB), scale(A, BC));
          else L = sub(scale(Cc, AB), scale(B, AC));
          out = scale(L, -I * (gs * gs));
          break;
        }
        default: break;
      }
      amput[id] = out;
      // propagator
      T K2 = mdot(Ks, Ks);
      if (is_vec(n.out)) {
        if (n.out == ZB) {
          Cx<T> den(K2 - T(cp.mz * cp.mz), T(cp.mz * cp.wz));
          Cx<T> KA = cdot(mom_to_vec(Ks), out);
          Vec4<T> v;
          for (int mu = 0; mu < 4; ++mu) v[mu] = out[mu] - KA * (Ks[mu] / T(cp.mz * cp.mz));
          cur[id] = scale(v, -I / den);
        } else {
          cur[id] = scale(out, -I / Cx<T>(K2));
        }
      } else {
        double m = cp.fmass(n.out), w = cp.width(n.out);
        Cx<T> den(K2 - T(m * m), T(m * w));
        Mat4<T> num;
        Mom<T> q = Ks;
        if (is_col(n.out)) for (auto& x : q) x = -x;  // momentum along the fermion arrow
        num = slash(mom_to_vec(q));
        for (int i = 0; i < 4; ++i) num[i][i] += Cx<T>(T(m));
        Cx<T> f = I / den;
        Vec4<T> v = is_row(n.out) ? row_mat(out, num) : mat_col(num, out);
        cur[id] = scale(v, f);
      }
    }
  }

  Cx<T> close(int amp_node, const std::vector<Mom<T>>& p, const std::vector<int>& hel) {
    int nl = (int)tp.proc.legs.size();
    Vec4<T> wr = external(nl - 1, p[nl - 1], hel[nl - 1]);
    const Vec4<T>& o = amput[amp_node];
    Line rl = tp.proc.legs[nl - 1].line;
    if (is_vec(rl)) return cdot(o, wr);
    return row_col(is_row(rl) ? wr : o, is_row(rl) ? o : wr);
  }
};

// |M|^2 summed over colours for one helicity; optionally the per-diagram amplitudes
template <class T>
T me_one_helicity(const Topology& tp, Eval<T>& ev, const std::vector<Mom<T>>& p, const std::vector<int>& hel,
                  std::vector<Cx<T>>* amps_out = nullptr) {
  ev.run(p, hel);
  size_t na = tp.amps.size();
  std::vector<Cx<T>> a(na);
  for (size_t d = 0; d < na; ++d) a[d] = ev.close(tp.amps[d], p, hel);
  if (amps_out) *amps_out = a;
  // sum_{d,e} a_d conj(a_e) CC_de  (real)
  T s(0.0);
  for (size_t d = 0; d < na; ++d) {
    Cx<T> row;
    for (size_t e = 0; e < na; ++e) {
      const C& c = tp.cc[d][e];
      if (c == C(0)) continue;
      row += cmul(c, conj(a[e]));
    }
    Cx<T> t = a[d] * row;
    s += t.re;
  }
  return s;
}

template <class T>
T me_event(const Topology& tp, const Couplings& cp, const std::vector<Mom<T>>& p, T* per_hel) {
  int nl = (int)tp.proc.legs.size();
  int nh = 1 << nl;
  Eval<T> ev(tp, cp);
  T tot(0.0);
  double norm = 1.0 / (tp.proc.hel_avg * tp.proc.col_avg * tp.proc.sym);
  std::vector<int> hel(nl);
  for (int h = 0; h < nh; ++h) {
    for (int i = 0; i < nl; ++i) hel[i] = ((h >> (nl - 1 - i)) & 1) ? +1 : -1;
    T v = me_one_helicity(tp, ev, p, hel) * T(norm);
    if (per_hel) per_hel[h] = v;
    tot += v;
  }
  return tot;
}

// ----------------------------------------------------------------------------
// RAMBO (Kleiss, Stirling, Ellis 1986): n massless momenta uniformly
// distributed in phase space, then rescaled to the final-state masses.
// Beams are massless along +z (first leg) and -z (second leg).
// Random-number usage for final particle i: rows 4i..4i+3 =
// (cos theta, phi, and the two factors of the energy -log(r3 r4)).
// ----------------------------------------------------------------------------
template <class T>
bool rambo(int nfin, double ecm, const double* fmass, const T* r /* 4*nfin */, Mom<T>* pout, T& wgt) {
  std::vector<Mom<T>> q(nfin);
  const double twopi = 2.0 * M_PI;
  for (int i = 0; i < nfin; ++i) {
    T c = T(2.0) * r[4 * i] - T(1.0);
    T s = sqrt(T(1.0) - c * c);
    T f = T(twopi) * r[4 * i + 1];
    T e = -log(r[4 * i + 2] * r[4 * i + 3]);
    q[i] = {e, e * s * cos(f), e * s * sin(f), e * c};
  }
  Mom<T> Q = {T(0.0), T(0.0), T(0.0), T(0.0)};
  for (int i = 0; i < nfin; ++i) for (int mu = 0; mu < 4; ++mu) Q[mu] += q[i][mu];
  T M = sqrt(mdot(Q, Q));
  T b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  T g = Q[0] / M;
  T a = T(1.0) / (T(1.0) + g);
  T x = T(ecm) / M;
  for (int i = 0; i < nfin; ++i) {
    T bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
    pout[i][0] = x * (g * q[i][0] + bq);
    for (int k = 0; k < 3; ++k) pout[i][k + 1] = x * (q[i][k + 1] + b[k] * q[i][0] + a * bq * b[k]);
  }
  // flat massless volume (no 2 pi factors)
  double fact = 1.0;
  for (int k = 2; k <= nfin - 1; ++k) fact *= k;          // (n-1)!
  double fact2 = 1.0;
  for (int k = 2; k <= nfin - 2; ++k) fact2 *= k;         // (n-2)!
  double w0 = std::pow(M_PI / 2.0, nfin - 1) * std::pow(ecm * ecm, nfin - 2) / (fact * fact2);
  wgt = T(w0);
  double msum = 0.0; bool massive = false;
  for (int i = 0; i < nfin; ++i) { msum += fmass[i]; if (fmass[i] != 0.0) massive = true; }
  if (!massive) return true;
  if (msum >= ecm) return false;
  // solve sum_i sqrt(m_i^2 + xi^2 E_i^2) = ecm by Newton's method
  T xi = T(std::sqrt(1.0 - (msum / ecm) * (msum / ecm)));
  int extra = 0;
  for (int it = 0; it < 50; ++it) {
    T f(-ecm), df(0.0);
    for (int i = 0; i < nfin; ++i) {
      T e = sqrt(T(fmass[i] * fmass[i]) + xi * xi * pout[i][0] * pout[i][0]);
      f += e;
      df += xi * pout[i][0] * pout[i][0] / e;
    }
    xi = xi - f / df;
    if (std::abs(val(f)) <= 1e-15 * ecm) { if (++extra >= 2) break; }
  }
  T w2(1.0), w3(0.0);
  for (int i = 0; i < nfin; ++i) {
    T kk = xi * pout[i][0];                           // |k_i| = xi |p_i| for massless p_i
    T e = sqrt(T(fmass[i] * fmass[i]) + kk * kk);
    for (int k = 1; k < 4; ++k) pout[i][k] = xi * pout[i][k];
    pout[i][0] = e;
    w2 = w2 * (kk / e);
    w3 += kk * kk / e;
  }
  T xin = xi;
  T pw(1.0);
  for (int k = 0; k < 2 * nfin - 3; ++k) pw = pw * xin;
  wgt = wgt * pw * w2 / w3 * T(ecm);
  return true;
}

template <class T>
bool event_momenta(const Process& P, const Couplings& cp, double ecm, const T* r, std::vector<Mom<T>>& p, T& wgt) {
  int nl = (int)P.legs.size();
  p.assign(nl, Mom<T>());
  double h = ecm / 2.0;
  p[0] = {T(h), T(0.0), T(0.0), T(h)};
  p[1] = {T(h), T(0.0), T(0.0), T(-h)};
  int nfin = nl - 2;
  std::vector<double> fm(nfin);
  for (int i = 0; i < nfin; ++i) fm[i] = cp.mass(P.legs[2 + i].mass_id);
  return rambo(nfin, ecm, fm.data(), r, &p[2], wgt);
}

static void parallel_for(long n, int nthreads, const std::function<void(long, long)>& fn) {
  if (nthreads <= 1 || n < 2) { fn(0, n); return; }
  std::vector<std::thread> th;
  long chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    long a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back(fn, a, b);
  }
  for (auto& x : th) x.join();
}

}  // namespace orc

// ----------------------------------------------------------------------------
// Colour flows (Sec. 2, colour-flow method).  The full-colour amplitude of one
// helicity, M(c) = sum_d a_d x_d(c) over the explicit colour assignments c of
// all legs, is written in the basis of the colour chains
//   chi_s(c) = (T^{a_{g(s_1)}} ... T^{a_{g(s_k)}})_{i_top j_antitop},
// g = the gluon legs in leg order, s the k! permutations in lexicographic
// order (one flow, chi = 1, without colour): M = sum_s J_s chi_s.  The
// coefficient of each amplitude on each chain is the projection
// P = G^{-1} B^dagger X with B[c][s] = chi_s(c), G = B^dagger B and
// X[c][d] = x_d(c); the residual max |B P - X| shows that every diagram's
// colour tensor lies in the span of the chains.
// ----------------------------------------------------------------------------
namespace orc {

struct FlowProjection {
  int nflow = 0;
  std::vector<C> P;  // [s][d]
  double residual = 0.0;
};

static FlowProjection* build_flow_projection(const Topology& tp) {
  const auto& legs = tp.proc.legs;
  const int nl = (int)legs.size();
  std::vector<int> g;
  int top = -1, atop = -1;
  for (int l = 0; l < nl; ++l) {
    if (legs[l].line == GLU) g.push_back(l);
    if (legs[l].line == ROW_T) top = l;
    if (legs[l].line == COL_T) atop = l;
  }
  const int ng = (int)g.size();
  std::vector<std::vector<int>> perms;
  std::vector<int> pm(ng);
  for (int i = 0; i < ng; ++i) pm[i] = i;
  do perms.push_back(pm); while (std::next_permutation(pm.begin(), pm.end()));
  const int nf = top >= 0 ? (int)perms.size() : 1;
  size_t ncol = 1;
  for (int l = 0; l < nl; ++l) ncol *= colour_dim(legs[l].line);
  const SU3& G3 = su3();
  // B[c][s]
  std::vector<C> B(ncol * nf, C(0));
  std::vector<int> col(nl);
  for (size_t A = 0; A < ncol; ++A) {
    size_t rem = A;
    for (int l = nl - 1; l >= 0; --l) { int d = colour_dim(legs[l].line); col[l] = (int)(rem % d); rem /= d; }
    if (top < 0) { B[A] = 1.0; continue; }
    for (int s = 0; s < nf; ++s) {
      C M[3][3];
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) M[i][j] = i == j ? 1.0 : 0.0;
      for (int k = 0; k < ng; ++k) {
        const int a = col[g[perms[s][k]]];
        C R[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            R[i][j] = 0;
            for (int m = 0; m < 3; ++m) R[i][j] += M[i][m] * G3.T[a][m][j];
          }
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) M[i][j] = R[i][j];
      }
      B[A * nf + s] = M[col[top]][col[atop]];
    }
  }
  const int na = (int)tp.amps.size();
  // normal equations G P = H, H = B^dagger X
  std::vector<C> Gm(nf * nf, C(0)), H((size_t)nf * na, C(0));
  for (size_t A = 0; A < ncol; ++A)
    for (int s = 0; s < nf; ++s) {
      const C b = std::conj(B[A * nf + s]);
      if (b == C(0)) continue;
      for (int t = 0; t < nf; ++t) Gm[s * nf + t] += b * B[A * nf + t];
      for (int d = 0; d < na; ++d) {
        const C x = tp.ctensor[tp.amps[d]][A];
        if (x != C(0)) H[(size_t)s * na + d] += b * x;
      }
    }
  // Gauss-Jordan elimination with partial pivoting on [G | H]
  for (int k = 0; k < nf; ++k) {
    int piv = k;
    for (int r = k + 1; r < nf; ++r) if (std::abs(Gm[r * nf + k]) > std::abs(Gm[piv * nf + k])) piv = r;
    if (piv != k) {
      for (int t = 0; t < nf; ++t) std::swap(Gm[k * nf + t], Gm[piv * nf + t]);
      for (int d = 0; d < na; ++d) std::swap(H[(size_t)k * na + d], H[(size_t)piv * na + d]);
    }
    const C inv = 1.0 / Gm[k * nf + k];
    for (int t = 0; t < nf; ++t) Gm[k * nf + t] *= inv;
    for (int d = 0; d < na; ++d) H[(size_t)k * na + d] *= inv;
    for (int r = 0; r < nf; ++r) {
      if (r == k) continue;
      const C f = Gm[r * nf + k];
      if (f == C(0)) continue;
      for (int t = 0; t < nf; ++t) Gm[r * nf + t] -= f * Gm[k * nf + t];
      for (int d = 0; d < na; ++d) H[(size_t)r * na + d] -= f * H[(size_t)k * na + d];
    }
  }
  auto* fp = new FlowProjection();
  fp->nflow = nf;
  fp->P = H;
  double res = 0.0;
  for (size_t A = 0; A < ncol; ++A)
    for (int d = 0; d < na; ++d) {
      C v = -tp.ctensor[tp.amps[d]][A];
      for (int s = 0; s < nf; ++s) v += B[A * nf + s] * H[(size_t)s * na + d];
      res = std::max(res, std::abs(v));
    }
  fp->residual = res;
  return fp;
}

static const FlowProjection* flow_projection(int proc) {
  static std::mutex mu;
  static FlowProjection* cache[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  Topology* tp = topology(proc);
  if (!tp) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[proc]) cache[proc] = build_flow_projection(*tp);
  return cache[proc];
}

}  // namespace orc

// ----------------------------------------------------------------------------
// C entry points (ctypes).  Arrays are structure-of-arrays with the event
// index fastest: rnd[k*nevt + i], mom[((p*4)+mu)*nevt + i].
// Return 0 on success, a negative number on a bad argument.
// ----------------------------------------------------------------------------
using namespace orc;
extern "C" {

int oracle_process_info(int proc, int* npar, int* nhel, int* ndiag, int* namp) {
  Topology* tp = topology(proc);
  if (!tp) return -2;
  *npar = (int)tp->proc.legs.size();
  *nhel = 1 << *npar;
  *ndiag = tp->ndiagrams;
  *namp = (int)tp->amps.size();
  return 0;
}

int oracle_rambo(int proc, long nevt, double ecm, const double* rnd, int nrows, const oracle_params* prm,
                 double* mom, double* wgt) {
  Process P = make_process(proc);
  if (P.legs.empty()) return -2;
  int nl = (int)P.legs.size();
  if (nrows < 4 * (nl - 2) || nevt < 0) return -1;
  Couplings cp = couplings(*prm);
  for (long i = 0; i < nevt; ++i) {
    double r[64];
    for (int k = 0; k < 4 * (nl - 2); ++k) r[k] = rnd[k * nevt + i];
    std::vector<Mom<double>> p; double w;
    if (!event_momenta(P, cp, ecm, r, p, w)) return -1;
    for (int a = 0; a < nl; ++a) for (int mu = 0; mu < 4; ++mu) mom[(a * 4 + mu) * nevt + i] = p[a][mu];
    wgt[i] = w;
  }
  return 0;
}

// me[i] (and per-helicity contributions me_hel[h*nevt + i] if non-null)
int oracle_me(int proc, long nevt, const double* mom, const oracle_params* prm, double* me, double* me_hel,
              int nthreads) {
  Topology* tp = topology(proc);
  if (!tp) return -2;
  if (nevt < 0) return -1;
  Couplings cp = couplings(*prm);
  int nl = (int)tp->proc.legs.size();
  int nh = 1 << nl;
  parallel_for(nevt, nthreads, [&](long a, long b) {
    std::vector<double> ph(nh);
    for (long i = a; i < b; ++i) {
      std::vector<Mom<double>> p(nl);
      for (int l = 0; l < nl; ++l) for (int mu = 0; mu < 4; ++mu) p[l][mu] = mom[(l * 4 + mu) * nevt + i];
      me[i] = me_event<double>(*tp, cp, p, ph.data());
      if (me_hel) for (int h = 0; h < nh; ++h) me_hel[(long)h * nevt + i] = ph[h];
    }
  });
  return 0;
}

// Per-diagram amplitudes for one event and one helicity (index h), in the
// order of the enumeration; returns the number written (<= cap).
int oracle_amplitudes(int proc, const double* mom1 /* [npar][4] */, int h, const oracle_params* prm,
                      const double* pol_override /* [8]: re/im of a vector replacing leg `pol_leg`, or null */,
                      int pol_leg, double* amps_reim, int cap) {
  Topology* tp = topology(proc);
  if (!tp) return -2;
  Couplings cp = couplings(*prm);
  int nl = (int)tp->proc.legs.size();
  std::vector<Mom<double>> p(nl);
  for (int l = 0; l < nl; ++l) for (int mu = 0; mu < 4; ++mu) p[l][mu] = mom1[l * 4 + mu];
  std::vector<int> hel(nl);
  for (int i = 0; i < nl; ++i) hel[i] = ((h >> (nl - 1 - i)) & 1) ? +1 : -1;
  Eval<double> ev(*tp, cp);
  if (pol_override && pol_leg >= 0 && pol_leg < nl) {
    ev.ov_leg = pol_leg;
    for (int mu = 0; mu < 4; ++mu) ev.ov_val[mu] = Cx<double>(pol_override[2 * mu], pol_override[2 * mu + 1]);
  }
  ev.run(p, hel);
  int na = (int)tp->amps.size();
  int nw = na < cap ? na : cap;
  for (int d = 0; d < nw; ++d) {
    Cx<double> a = ev.close(tp->amps[d], p, hel);
    amps_reim[2 * d] = a.re; amps_reim[2 * d + 1] = a.im;
  }
  return nw;
}

// Sum over colours of a_d conj(a_e) CC_de for given amplitudes (tests of the colour Gram matrix)
int oracle_colour_gram(int proc, double* cc_reim, int cap) {
  Topology* tp = topology(proc);
  if (!tp) return -2;
  int na = (int)tp->amps.size();
  if ((long)na * na > cap) return -1;
  for (int d = 0; d < na; ++d)
    for (int e = 0; e < na; ++e) { cc_reim[2 * (d * na + e)] = tp->cc[d][e].real(); cc_reim[2 * (d * na + e) + 1] = tp->cc[d][e].imag(); }
  return na;
}

// Chain-basis colour matrix C_{sigma tau} = sum over colours of
// (T^{a_s1}..T^{a_sn})_{ij} conj((T^{a_t1}..T^{a_tn})_{ij}) for n gluons, with the
// n! permutations in lexicographic order; explicit SU(3) sums.
int oracle_chain_colour_matrix(int ng, double* out_reim, int cap) {
  if (ng < 1 || ng > 4) return -1;
  std::vector<std::vector<int>> perms;
  std::vector<int> p(ng); for (int i = 0; i < ng; ++i) p[i] = i;
  do perms.push_back(p); while (std::next_permutation(p.begin(), p.end()));
  int nf = (int)perms.size();
  if (nf * nf > cap) return -1;
  const SU3& G = su3();
  int ncol = 1; for (int i = 0; i < ng; ++i) ncol *= 8;
  // chains[s][colour assignment][i][j]
  std::vector<std::vector<C>> ch(nf, std::vector<C>((size_t)ncol * 9, C(0)));
  for (int s = 0; s < nf; ++s)
    for (int A = 0; A < ncol; ++A) {
      int a[4]; int rem = A;
      for (int k = ng - 1; k >= 0; --k) { a[k] = rem % 8; rem /= 8; }
      C M[3][3];
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) M[i][j] = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < ng; ++k) {
        int g = a[perms[s][k]];
        C R[3][3];
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) { R[i][j] = 0; for (int l = 0; l < 3; ++l) R[i][j] += M[i][l] * G.T[g][l][j]; }
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) M[i][j] = R[i][j];
      }
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) ch[s][(size_t)A * 9 + i * 3 + j] = M[i][j];
    }
  for (int s = 0; s < nf; ++s)
    for (int t = 0; t < nf; ++t) {
      C acc = 0;
      for (size_t k = 0; k < ch[s].size(); ++k) acc += ch[s][k] * std::conj(ch[t][k]);
      out_reim[2 * (s * nf + t)] = acc.real(); out_reim[2 * (s * nf + t) + 1] = acc.imag();
    }
  return nf;
}

// SU(3) generators and structure constants (tests)
int oracle_su3(double* T_reim /* 8*3*3*2 */, double* f /* 512 */) {
  const SU3& G = su3();
  for (int a = 0; a < 8; ++a) for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
    T_reim[2 * ((a * 3 + i) * 3 + j)] = G.T[a][i][j].real();
    T_reim[2 * ((a * 3 + i) * 3 + j) + 1] = G.T[a][i][j].imag();
  }
  for (int k = 0; k < 512; ++k) f[k] = (&G.f[0][0][0])[k];
  return 0;
}

// External wavefunctions (tests of the spinor / polarisation identities).
// kind: 0 u, 1 v, 2 eps (incoming), returns 4 complex components
int oracle_wavefunction(int kind, const double* p4, double m, int lam, double* out_reim) {
  Mom<double> p = {p4[0], p4[1], p4[2], p4[3]};
  Vec4<double> w;
  if (kind == 0) w = spinor_u(p, m, lam);
  else if (kind == 1) w = spinor_v(p, m, lam);
  else if (kind == 2) w = polvec(p, lam);
  else return -1;
  for (int k = 0; k < 4; ++k) { out_reim[2 * k] = w[k].re; out_reim[2 * k + 1] = w[k].im; }
  return 0;
}
int oracle_gamma(double* g_reim /* 5*4*4*2: gamma^0..3, gamma5 */) {
  const Dirac& D = dirac();
  for (int m = 0; m < 5; ++m) for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) {
    std::complex<double> v = m < 4 ? D.g[m][i][j] : D.g5[i][j];
    g_reim[2 * ((m * 4 + i) * 4 + j)] = v.real(); g_reim[2 * ((m * 4 + i) * 4 + j) + 1] = v.imag();
  }
  return 0;
}

// Gradient of me with respect to the random numbers (forward-mode dual
// numbers through RAMBO and the amplitudes).  grad[k*nevt + i] for k < nrows;
// rows RAMBO does not consume get exactly zero.
int oracle_me_grad(int proc, long nevt, double ecm, const double* rnd, int nrows, const oracle_params* prm,
                   double* me, double* grad, int nthreads) {
  Topology* tp = topology(proc);
  if (!tp) return -2;
  int nl = (int)tp->proc.legs.size();
  int nused = 4 * (nl - 2);
  if (nrows < nused || nused > ND) return -1;
  Couplings cp = couplings(*prm);
  int bad = 0;
  parallel_for(nevt, nthreads, [&](long a, long b) {
    for (long i = a; i < b; ++i) {
      std::vector<Dual> r(nused);
      for (int k = 0; k < nused; ++k) { r[k] = Dual(rnd[(long)k * nevt + i]); r[k].d[k] = 1.0; }
      std::vector<Mom<Dual>> p; Dual w;
      if (!event_momenta(tp->proc, cp, ecm, r.data(), p, w)) { bad = 1; continue; }
      Dual m = me_event<Dual>(*tp, cp, p, nullptr);
      me[i] = m.v;
      for (int k = 0; k < nrows; ++k) grad[(long)k * nevt + i] = k < nused ? m.d[k] : 0.0;
    }
  });
  return bad ? -1 : 0;
}

// Event accumulation: out[0] = sum w*me, out[1] = sum (w*me)^2, out[2] = N (pairwise summation)
static void pairwise(const double* me, const double* w, long a, long b, double& s1, double& s2) {
  if (b - a <= 8) {
    s1 = 0; s2 = 0;
    for (long i = a; i < b; ++i) { double x = me[i] * w[i]; s1 += x; s2 += x * x; }
    return;
  }
  long m = a + (b - a) / 2;
  double l1, l2, r1, r2;
  pairwise(me, w, a, m, l1, l2);
  pairwise(me, w, m, b, r1, r2);
  s1 = l1 + r1; s2 = l2 + r2;
}
int oracle_event_sum(long nevt, const double* me, const double* w, double* out3) {
  if (nevt < 0) return -1;
  double s1 = 0, s2 = 0;
  if (nevt > 0) pairwise(me, w, 0, nevt, s1, s2);
  out3[0] = s1; out3[1] = s2; out3[2] = (double)nevt;
  return 0;
}

// Colour-flow decomposition: number of flows and the projection residual
int oracle_colour_flow_info(int proc, int* nflow, double* residual) {
  const FlowProjection* fp = flow_projection(proc);
  if (!fp) return -2;
  *nflow = fp->nflow;
  *residual = fp->residual;
  return 0;
}

// Colour-flow amplitudes J_s of every helicity h (index as in oracle_me):
// jf[((h*nflow + s)*nevt + i)*2 + {0: re, 1: im}], without the average factors
int oracle_colour_flows(int proc, long nevt, const double* mom, const oracle_params* prm, double* jf, int nthreads) {
  Topology* tp = topology(proc);
  const FlowProjection* fp = flow_projection(proc);
  if (!tp || !fp) return -2;
  if (nevt < 0) return -1;
  Couplings cp = couplings(*prm);
  const int nl = (int)tp->proc.legs.size(), nh = 1 << nl, nf = fp->nflow, na = (int)tp->amps.size();
  parallel_for(nevt, nthreads, [&](long a, long b) {
    Eval<double> ev(*tp, cp);
    std::vector<int> hel(nl);
    std::vector<Cx<double>> amp(na);
    for (long i = a; i < b; ++i) {
      std::vector<Mom<double>> p(nl);
      for (int l = 0; l < nl; ++l) for (int mu = 0; mu < 4; ++mu) p[l][mu] = mom[(l * 4 + mu) * nevt + i];
      for (int h = 0; h < nh; ++h) {
        for (int k = 0; k < nl; ++k) hel[k] = ((h >> (nl - 1 - k)) & 1) ? +1 : -1;
        ev.run(p, hel);
        for (int d = 0; d < na; ++d) amp[d] = ev.close(tp->amps[d], p, hel);
        for (int s = 0; s < nf; ++s) {
          C j = 0;
          for (int d = 0; d < na; ++d) j += fp->P[(size_t)s * na + d] * C(amp[d].re, amp[d].im);
          const size_t o = (((size_t)h * nf + s) * nevt + i) * 2;
          jf[o] = j.real();
          jf[o + 1] = j.imag();
        }
      }
    }
  });
  return 0;
}

}  // extern "C"
