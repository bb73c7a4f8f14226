// Helicity-amplitude routines (Sec. 2: "external particle", "internal
// particle" and "amplitude" routines; names follow the routines the paper
// shows in Fig. 1).  All formulas are written out in the chiral (Weyl) basis,
//   gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]],  sigma^mu = (1, s),
//   sigmabar^mu = (1, -s),  gamma5 = diag(-1, -1, 1, 1),
// so that a slashed vector V/ = gamma^mu V_mu has the 2x2 blocks
//   sigma.V    = [[V0 - V3, -(V1 - i V2)], [-(V1 + i V2), V0 + V3]]  (upper right)
//   sigmabar.V = [[V0 + V3,   V1 - i V2 ], [  V1 + i V2 , V0 - V3]]  (lower left).
// Feynman rules (Peskin & Schroeder): quark-gluon vertex i g gamma^mu T^a,
// three-gluon vertex g f^abc [g^{mu nu}(k - p)^rho + ...] (momenta incoming),
// four-gluon vertex -i g^2 [...]; colour factors are handled by the colour-flow
// decomposition, these routines carry the colour-stripped Lorentz parts.
// Every internal-particle routine multiplies by a propagator factor `prop`
// (fermion: i / (K^2 - m^2 + i m Gamma), vector: -i / (K^2 - M^2 + i M Gamma)),
// which the caller forms once per event in FP64.
// All momenta K passed to vertices are outgoing sums of external momenta.
#pragma once
#include "mg_types.cuh"

namespace mg {

template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return 1.0f / sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }

// Helicity eigenspinor chi_lam(p^) of sigma.p^ (eigenvalue lam).  |p| + pz is
// formed as pT^2 / (|p| - pz) when pz < 0, so particles near -z keep full
// precision.
template <class R>
__device__ __forceinline__ void helicity_chi(const R* p, int lam, cx<R>& c0, cx<R>& c1) {
  const R px = p[1], py = p[2], pz = p[3];
  const R pt2 = px * px + py * py;
  const R pp = sqrt(pt2 + pz * pz);
  const R ppz = pz >= R(0) ? pp + pz : pt2 / (pp - pz);
  if (ppz <= R(0)) {  // exactly along -z
    if (lam > 0) { c0 = cx<R>(R(0), R(0)); c1 = cx<R>(R(1), R(0)); }
    else { c0 = cx<R>(R(-1), R(0)); c1 = cx<R>(R(0), R(0)); }
    return;
  }
  const R nrm = rsqrt_<R>(R(2) * pp * ppz);
  if (lam > 0) { c0 = cx<R>(ppz * nrm, R(0)); c1 = cx<R>(px * nrm, py * nrm); }
  else { c0 = cx<R>(-px * nrm, py * nrm); c1 = cx<R>(ppz * nrm, R(0)); }
}

// omega_+ = sqrt(E + |p|), omega_- = sqrt(E - |p|) = m / omega_+ (exactly 0 for m = 0)
template <class R>
__device__ __forceinline__ void omegas(const R* p, R m, R& wp, R& wm) {
  const R pp = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
  wp = sqrt(p[0] + pp);
  wm = m == R(0) ? R(0) : m / wp;
}

// Flowing-in fermion (column spinor): nsf = +1 incoming particle u(p, hel),
// nsf = -1 outgoing antiparticle v(p, hel).  p is the physical momentum.
//   u = (omega_{-hel} chi_hel, omega_{+hel} chi_hel)
//   v = (-hel omega_{+hel} chi_{-hel}, hel omega_{-hel} chi_{-hel})
template <class R>
__device__ __forceinline__ W4<R> ixxxxx(const R* p, R m, int hel, int nsf) {
  R wp, wm;
  omegas(p, m, wp, wm);
  cx<R> c0, c1;
  W4<R> f;
  if (nsf > 0) {
    helicity_chi(p, hel, c0, c1);
    const R lo = hel > 0 ? wm : wp, hi = hel > 0 ? wp : wm;
    f.w[0] = lo * c0; f.w[1] = lo * c1; f.w[2] = hi * c0; f.w[3] = hi * c1;
  } else {
    helicity_chi(p, -hel, c0, c1);
    const R a = hel > 0 ? -wp : wm, b = hel > 0 ? wm : -wp;
    f.w[0] = a * c0; f.w[1] = a * c1; f.w[2] = b * c0; f.w[3] = b * c1;
  }
  return f;
}

// Flowing-out fermion (row spinor psi^dagger gamma^0): nsf = +1 outgoing
// particle u-bar(p, hel), nsf = -1 incoming antiparticle v-bar(p, hel).
template <class R>
__device__ __forceinline__ W4<R> oxxxxx(const R* p, R m, int hel, int nsf) {
  const W4<R> c = ixxxxx<R>(p, m, hel, nsf);
  W4<R> f;
  f.w[0] = conj(c.w[2]); f.w[1] = conj(c.w[3]); f.w[2] = conj(c.w[0]); f.w[3] = conj(c.w[1]);
  return f;
}

// Massless vector boson: eps(k, hel) = (-hel e1 - i e2)/sqrt2 with
// e1 = (0, cos th cos ph, cos th sin ph, -sin th), e2 = (0, -sin ph, cos ph, 0);
// nsv = +1 incoming (eps), nsv = -1 outgoing (eps*).
template <class R>
__device__ __forceinline__ W4<R> vxxxxx(const R* k, int hel, int nsv) {
  const R kt = sqrt(k[1] * k[1] + k[2] * k[2]);
  const R kk = sqrt(kt * kt + k[3] * k[3]);
  R ct, st, cp, sp;
  if (kt == R(0)) { ct = k[3] >= R(0) ? R(1) : R(-1); st = R(0); cp = R(1); sp = R(0); }
  else { ct = k[3] / kk; st = kt / kk; cp = k[1] / kt; sp = k[2] / kt; }
  const R r2 = R(0.70710678118654752440);
  const R a = -R(hel) * r2;
  const R b = nsv > 0 ? -r2 : r2;  // imaginary part sign (conjugated for outgoing)
  W4<R> v;
  v.w[0] = cx<R>(R(0), R(0));
  v.w[1] = cx<R>(a * ct * cp, b * -sp);
  v.w[2] = cx<R>(a * ct * sp, b * cp);
  v.w[3] = cx<R>(-a * st, R(0));
  return v;
}

// ---- Dirac algebra helpers ------------------------------------------------
// row . V/   (V complex, upper index)
template <class R>
__device__ __forceinline__ W4<R> row_slash(const W4<R>& f, const W4<R>& V) {
  const cx<R> vp = V.w[0] + V.w[3], vm = V.w[0] - V.w[3];
  const cx<R> vxpy = V.w[1] + mul_i(V.w[2]), vxmy = V.w[1] - mul_i(V.w[2]);
  W4<R> o;
  o.w[0] = cfma(f.w[3], vxpy, f.w[2] * vp);
  o.w[1] = cfma(f.w[3], vm, f.w[2] * vxmy);
  o.w[2] = cfma(-f.w[1], vxpy, f.w[0] * vm);
  o.w[3] = cfma(-f.w[0], vxmy, f.w[1] * vp);
  return o;
}
// V/ . col
template <class R>
__device__ __forceinline__ W4<R> slash_col(const W4<R>& V, const W4<R>& f) {
  const cx<R> vp = V.w[0] + V.w[3], vm = V.w[0] - V.w[3];
  const cx<R> vxpy = V.w[1] + mul_i(V.w[2]), vxmy = V.w[1] - mul_i(V.w[2]);
  W4<R> o;
  o.w[0] = cfma(-vxmy, f.w[3], vm * f.w[2]);
  o.w[1] = cfma(-vxpy, f.w[2], vp * f.w[3]);
  o.w[2] = cfma(vxmy, f.w[1], vp * f.w[0]);
  o.w[3] = cfma(vm, f.w[1], vxpy * f.w[0]);
  return o;
}
// row . (K/ + m)  for a real momentum K
template <class R>
__device__ __forceinline__ W4<R> row_kslash_m(const W4<R>& f, const R* K, R m) {
  const R kp = K[0] + K[3], km = K[0] - K[3];
  const cx<R> kxpy(K[1], K[2]), kxmy(K[1], -K[2]);
  W4<R> o;
  o.w[0] = rfma(m, f.w[0], cfma(f.w[3], kxpy, kp * f.w[2]));
  o.w[1] = rfma(m, f.w[1], cfma(f.w[2], kxmy, km * f.w[3]));
  o.w[2] = rfma(m, f.w[2], cfma(-f.w[1], kxpy, km * f.w[0]));
  o.w[3] = rfma(m, f.w[3], cfma(-f.w[0], kxmy, kp * f.w[1]));
  return o;
}
// (-K/ + m) . col
template <class R>
__device__ __forceinline__ W4<R> mkslash_m_col(const R* K, R m, const W4<R>& f) {
  const R kp = K[0] + K[3], km = K[0] - K[3];
  const cx<R> kxpy(K[1], K[2]), kxmy(K[1], -K[2]);
  W4<R> o;
  o.w[0] = rfma(m, f.w[0], cfma(kxmy, f.w[3], -km * f.w[2]));
  o.w[1] = rfma(m, f.w[1], cfma(kxpy, f.w[2], -kp * f.w[3]));
  o.w[2] = rfma(m, f.w[2], cfma(-kxmy, f.w[1], -kp * f.w[0]));
  o.w[3] = rfma(m, f.w[3], cfma(-kxpy, f.w[0], -km * f.w[1]));
  return o;
}
template <class R>
__device__ __forceinline__ cx<R> row_col(const W4<R>& a, const W4<R>& b) {
  return cfma(a.w[3], b.w[3], cfma(a.w[2], b.w[2], cfma(a.w[1], b.w[1], a.w[0] * b.w[0])));
}
// Minkowski product of two complex vectors (no conjugation)
template <class R>
__device__ __forceinline__ cx<R> vdot(const W4<R>& a, const W4<R>& b) {
  return cfma(-a.w[3], b.w[3], cfma(-a.w[2], b.w[2], cfma(-a.w[1], b.w[1], a.w[0] * b.w[0])));
}
template <class R>
__device__ __forceinline__ cx<R> kdot(const R* k, const W4<R>& a) {
  return rfma(-k[3], a.w[3], rfma(-k[2], a.w[2], rfma(-k[1], a.w[1], k[0] * a.w[0])));
}
template <class R>
__device__ __forceinline__ W4<R> scale(const W4<R>& a, cx<R> s) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = a.w[k] * s;
  return o;
}
// row . gamma^mu (gl PL + gr PR) . col, upper index mu
template <class R>
__device__ __forceinline__ W4<R> bilinear(const W4<R>& f, const W4<R>& g, R gl, R gr) {
  // terms with g.w[0,1] (left) get gl, with g.w[2,3] (right) get gr
  const cx<R> a02 = f.w[0] * g.w[2], a13 = f.w[1] * g.w[3], a03 = f.w[0] * g.w[3], a12 = f.w[1] * g.w[2];
  const cx<R> b20 = f.w[2] * g.w[0], b31 = f.w[3] * g.w[1], b21 = f.w[2] * g.w[1], b30 = f.w[3] * g.w[0];
  W4<R> j;
  j.w[0] = gr * (a02 + a13) + gl * (b20 + b31);
  j.w[1] = gr * (a03 + a12) - gl * (b21 + b30);
  j.w[2] = mul_i(gr * (a12 - a03) + gl * (b21 - b30));
  j.w[3] = gr * (a02 - a13) + gl * (b31 - b20);
  return j;
}

// ---- amplitude routines -----------------------------------------------------
// i g  row . V/ . col  (fermion-fermion-vector vertex, vector coupling)
template <class R>
__device__ __forceinline__ cx<R> FFV1_0(const W4<R>& fo, const W4<R>& fi, const W4<R>& v, R g) {
  return mul_i(g * row_col(row_slash(fo, v), fi));
}
// -i gz row . V/ (gl PL + gr PR) . col  (Z vertex)
template <class R>
__device__ __forceinline__ cx<R> FFV2_4_0(const W4<R>& fo, const W4<R>& fi, const W4<R>& v, R gz, R gl, R gr) {
  W4<R> c = fi;
  c.w[0] = gl * c.w[0]; c.w[1] = gl * c.w[1]; c.w[2] = gr * c.w[2]; c.w[3] = gr * c.w[3];
  return mul_mi(gz * row_col(row_slash(fo, v), c));
}

// three-gluon amplitude, outgoing momenta K1..K3 of the three branches
// (incoming vertex momenta q = -K):
//   g [ (A1.A2)((q1 - q2).A3) + (A2.A3)((q2 - q3).A1) + (A3.A1)((q3 - q1).A2) ]
template <class R>
__device__ __forceinline__ cx<R> VVV1_0(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, const R* K1, const R* K2,
                                        const R* K3, R g) {
  R d12[4], d23[4], d31[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    d12[mu] = K2[mu] - K1[mu];
    d23[mu] = K3[mu] - K2[mu];
    d31[mu] = K1[mu] - K3[mu];
  }
  return g * (vdot(a1, a2) * kdot(d12, a3) + vdot(a2, a3) * kdot(d23, a1) + vdot(a3, a1) * kdot(d31, a2));
}
// four-gluon amplitude, Lorentz term t (legs 0..3, colour f^{a0 a1 e} f^{a2 a3 e},
// f^{a0 a2 e} f^{a1 a3 e}, f^{a0 a3 e} f^{a1 a2 e} for t = 0, 1, 2):
//   -i g^2 [(A0.A2)(A1.A3) - (A0.A3)(A1.A2)],  [(A0.A1)(A2.A3) - (A0.A3)(A1.A2)],
//   [(A0.A1)(A2.A3) - (A0.A2)(A1.A3)]
template <class R>
__device__ __forceinline__ cx<R> VVVV_0(int t, const W4<R>& a0, const W4<R>& a1, const W4<R>& a2, const W4<R>& a3,
                                        R g2) {
  cx<R> l;
  if (t == 0) l = vdot(a0, a2) * vdot(a1, a3) - vdot(a0, a3) * vdot(a1, a2);
  else if (t == 1) l = vdot(a0, a1) * vdot(a2, a3) - vdot(a0, a3) * vdot(a1, a2);
  else l = vdot(a0, a1) * vdot(a2, a3) - vdot(a0, a2) * vdot(a1, a3);
  return mul_mi(g2 * l);
}

// ---- internal-particle routines ---------------------------------------------
// off-shell flowing-out fermion:  [row . (i g V/)] (K/ + m) prop,  K = outgoing momentum
template <class R>
__device__ __forceinline__ W4<R> FFV1_2(const W4<R>& fo, const W4<R>& v, R g, const R* K, R m, cx<R> prop) {
  return scale(row_kslash_m(row_slash(fo, v), K, m), mul_i(g * prop));
}
// off-shell flowing-in fermion:  (-K/ + m) [(i g V/) . col] prop
template <class R>
__device__ __forceinline__ W4<R> FFV1_1(const W4<R>& fi, const W4<R>& v, R g, const R* K, R m, cx<R> prop) {
  return scale(mkslash_m_col(K, m, slash_col(v, fi)), mul_i(g * prop));
}
// off-shell vector from a fermion pair:  i g (row . gamma^mu . col) prop
template <class R>
__device__ __forceinline__ W4<R> FFV1P0_3(const W4<R>& fo, const W4<R>& fi, R g, cx<R> prop) {
  return scale(bilinear(fo, fi, R(1), R(1)), mul_i(g * prop));
}
// off-shell Z from a lepton pair: -i gz (row . gamma^mu (gl PL + gr PR) . col) prop
template <class R>
__device__ __forceinline__ W4<R> FFV2_4_3(const W4<R>& fo, const W4<R>& fi, R gz, R gl, R gr, cx<R> prop) {
  return scale(bilinear(fo, fi, gl, gr), mul_mi(gz * prop));
}
// off-shell gluon from two gluons with outgoing momenta K1, K2 (incoming
// vertex momenta q1 = -K1, q2 = -K2, q3 = K1 + K2):
//   g [ (A1.A2)(q1 - q2) + A2 ((q2 - q3).A1) + A1 ((q3 - q1).A2) ] prop
template <class R>
__device__ __forceinline__ W4<R> VVV1P0_1(const W4<R>& a1, const W4<R>& a2, const R* K1, const R* K2, R g, cx<R> prop) {
  R d12[4], d23[4], d31[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    d12[mu] = K2[mu] - K1[mu];
    d23[mu] = -(K1[mu] + R(2) * K2[mu]);
    d31[mu] = R(2) * K1[mu] + K2[mu];
  }
  const cx<R> a12 = vdot(a1, a2);
  const cx<R> c1 = kdot(d23, a1);
  const cx<R> c2 = kdot(d31, a2);
  const cx<R> s = g * prop;
  W4<R> o;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) o.w[mu] = cfma(a1.w[mu], c2, cfma(a2.w[mu], c1, d12[mu] * a12)) * s;
  return o;
}
// four-gluon vertex, the three colour-stripped Lorentz terms (legs A1, A2, A3, new):
//   VVVV1P0_1: (A1.A3) A2 - (A2.A3) A1   with colour f^{a1 a2 e} f^{a3 new e}
//   VVVV3P0_1: (A1.A2) A3 - (A2.A3) A1   with colour f^{a1 a3 e} f^{a2 new e}
//   VVVV4P0_1: (A1.A2) A3 - (A1.A3) A2   with colour f^{a1 new e} f^{a2 a3 e}
// each times -i g^2 prop
template <class R>
__device__ __forceinline__ W4<R> vvvv_comb(const W4<R>& x, cx<R> cx_, const W4<R>& y, cx<R> cy, cx<R> s) {
  W4<R> o;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) o.w[mu] = cfma(-cy, y.w[mu], cx_ * x.w[mu]) * s;
  return o;
}
template <class R>
__device__ __forceinline__ W4<R> VVVV1P0_1(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, R g2, cx<R> prop) {
  return vvvv_comb(a2, vdot(a1, a3), a1, vdot(a2, a3), mul_mi(g2 * prop));
}
template <class R>
__device__ __forceinline__ W4<R> VVVV3P0_1(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, R g2, cx<R> prop) {
  return vvvv_comb(a3, vdot(a1, a2), a1, vdot(a2, a3), mul_mi(g2 * prop));
}
template <class R>
__device__ __forceinline__ W4<R> VVVV4P0_1(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, R g2, cx<R> prop) {
  return vvvv_comb(a3, vdot(a1, a2), a2, vdot(a1, a3), mul_mi(g2 * prop));
}

// ---- amputated currents ------------------------------------------------------
// The vertex of an amplitude with one operand Y left out and no propagator, so
// that the amplitude is the plain contraction sum_i X_i Y_i (dot4).  Spinors:
// the row / column spinor of the vertex; vectors: LOWER index (metric applied).
// i g row . V/   (pairs with a column spinor)
template <class R>
__device__ __forceinline__ W4<R> FFV1_2A(const W4<R>& fo, const W4<R>& v, R g) {
  W4<R> o = row_slash(fo, v);
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = mul_i(g * o.w[k]);
  return o;
}
// i g V/ . col   (pairs with a row spinor)
template <class R>
__device__ __forceinline__ W4<R> FFV1_1A(const W4<R>& fi, const W4<R>& v, R g) {
  W4<R> o = slash_col(v, fi);
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = mul_i(g * o.w[k]);
  return o;
}
// i g (row . gamma_mu . col)
template <class R>
__device__ __forceinline__ W4<R> FFV1P0_3A(const W4<R>& fo, const W4<R>& fi, R g) {
  const W4<R> j = bilinear(fo, fi, R(1), R(1));
  W4<R> o;
  o.w[0] = mul_i(g * j.w[0]);
#pragma unroll
  for (int k = 1; k < 4; ++k) o.w[k] = mul_mi(g * j.w[k]);
  return o;
}
// -i gz (row . gamma_mu (gl PL + gr PR) . col)
template <class R>
__device__ __forceinline__ W4<R> FFV2_4_3A(const W4<R>& fo, const W4<R>& fi, R gz, R gl, R gr) {
  const W4<R> j = bilinear(fo, fi, gl, gr);
  W4<R> o;
  o.w[0] = mul_mi(gz * j.w[0]);
#pragma unroll
  for (int k = 1; k < 4; ++k) o.w[k] = mul_i(gz * j.w[k]);
  return o;
}
// g [ (A1.A2)(q1 - q2)_mu + A2_mu ((q2 - q3).A1) + A1_mu ((q3 - q1).A2) ],
// q1 = -K1, q2 = -K2, q3 = K1 + K2 (as VVV1P0_1)
template <class R>
__device__ __forceinline__ W4<R> VVV1P0_1A(const W4<R>& a1, const W4<R>& a2, const R* K1, const R* K2, R g) {
  R d12[4], d23[4], d31[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    d12[mu] = K2[mu] - K1[mu];
    d23[mu] = -(K1[mu] + R(2) * K2[mu]);
    d31[mu] = R(2) * K1[mu] + K2[mu];
  }
  const cx<R> a12 = vdot(a1, a2);
  const cx<R> c1 = kdot(d23, a1);
  const cx<R> c2 = kdot(d31, a2);
  W4<R> o;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const cx<R> n = cfma(a1.w[mu], c2, cfma(a2.w[mu], c1, d12[mu] * a12));
    o.w[mu] = (mu == 0 ? g : -g) * n;
  }
  return o;
}
// -i g^2 [ (x . (..)) - (y . (..)) ] of one four-gluon term (see vvvv_comb)
template <class R>
__device__ __forceinline__ W4<R> vvvv_comb_a(const W4<R>& x, cx<R> cx_, const W4<R>& y, cx<R> cy, R g2) {
  W4<R> o;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const cx<R> t = cfma(-cy, y.w[mu], cx_ * x.w[mu]);
    o.w[mu] = mu == 0 ? mul_mi(g2 * t) : mul_i(g2 * t);
  }
  return o;
}
// s + y, s - y, s + i y, s - i y (sums of left-out operands with a common phase)
template <class R>
__device__ __forceinline__ W4<R> w4_add(const W4<R>& s, const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = s.w[k] + y.w[k];
  return o;
}
template <class R>
__device__ __forceinline__ W4<R> w4_sub(const W4<R>& s, const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = s.w[k] - y.w[k];
  return o;
}
template <class R>
__device__ __forceinline__ W4<R> w4_addi(const W4<R>& s, const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = s.w[k] + mul_i(y.w[k]);
  return o;
}
template <class R>
__device__ __forceinline__ W4<R> w4_subi(const W4<R>& s, const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = s.w[k] - mul_i(y.w[k]);
  return o;
}
// contraction of an amputated current with the left-out operand, the real and
// imaginary parts each one chain of fused multiply-adds (16 operations)
#ifndef MG_DOT4_PAIRS
// FP32 contractions in paired FP32 instructions: bit 0 those accumulated
// straight into one colour flow, bit 1 the others (their extra registers made
// the gg -> t t~ g g kernel spill), bit 2 the additions of an amplitude into
// its several colour flows
#define MG_DOT4_PAIRS 5
#endif
// FP32 form: P = sum (xr yr, xi yi) and Q = sum (xi yr, xr yi) side by side in
// the paired FP32 instructions (8 FFMA2), Re = P.x - P.y, Im = Q.x + Q.y; the
// initial pairs carry a value the result is added to
__device__ __forceinline__ void dot4_pairs(const W4<float>& x, const W4<float>& y, float2& p, float2& q) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 yk = make_float2(y.w[k].re, y.w[k].im);
    p = __ffma2_rn(make_float2(x.w[k].re, x.w[k].im), yk, p);
    q = __ffma2_rn(make_float2(x.w[k].im, x.w[k].re), yk, q);
  }
}

template <class R>
__device__ __forceinline__ cx<R> dot4(const W4<R>& x, const W4<R>& y) {
  if constexpr (sizeof(R) == 4 && (MG_DOT4_PAIRS & 2)) {
    float2 p = make_float2(0.0f, 0.0f), q = make_float2(0.0f, 0.0f);
    dot4_pairs(x, y, p, q);
    return cx<R>(p.x - p.y, q.x + q.y);
  }
  R re = x.w[0].re * y.w[0].re, im = x.w[0].re * y.w[0].im;
  re = fmac(-x.w[0].im, y.w[0].im, re);
  im = fmac(x.w[0].im, y.w[0].re, im);
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    re = fmac(x.w[k].re, y.w[k].re, re);
    re = fmac(-x.w[k].im, y.w[k].im, re);
    im = fmac(x.w[k].re, y.w[k].im, im);
    im = fmac(x.w[k].im, y.w[k].re, im);
  }
  return cx<R>(re, im);
}

// J += i^PH a (PH 0: +1, 1: -1, 2: +i, 3: -i) for an amplitude that feeds
// several flows; FP32 with bit 2 of MG_DOT4_PAIRS: one paired FP32 add or FMA
// with a constant phase pair
template <int PH, class R>
__device__ __forceinline__ void flow_add(cx<R>& J, cx<R> a) {
  if constexpr (sizeof(R) == 4 && (MG_DOT4_PAIRS & 4)) {
    float2 j = make_float2(J.re, J.im);
    if constexpr (PH == 0) j = __fadd2_rn(j, make_float2(a.re, a.im));
    else if constexpr (PH == 1) j = __ffma2_rn(make_float2(-1.0f, -1.0f), make_float2(a.re, a.im), j);
    else if constexpr (PH == 2) j = __ffma2_rn(make_float2(-1.0f, 1.0f), make_float2(a.im, a.re), j);
    else j = __ffma2_rn(make_float2(1.0f, -1.0f), make_float2(a.im, a.re), j);
    J.re = j.x;
    J.im = j.y;
    return;
  }
  if constexpr (PH == 0) J += a;
  else if constexpr (PH == 1) J -= a;
  else if constexpr (PH == 2) J += mul_i(a);
  else J -= mul_i(a);
}

// J += i^PH sum_i X_i Y_i straight into one colour flow (PH 0: +1, 1: -1,
// 2: +i, 3: -i): the chains start from the flow's value, no separate add
template <int PH, class R>
__device__ __forceinline__ void dot4_acc(cx<R>& J, const W4<R>& x, const W4<R>& y) {
  if constexpr (sizeof(R) == 4 && (MG_DOT4_PAIRS & 1)) {
    // Re(XY) = P.x - P.y, Im(XY) = Q.x + Q.y, each started from the flow's part
    float2 p, q;
    if constexpr (PH == 0) { p = make_float2(J.re, 0.0f); q = make_float2(J.im, 0.0f); }
    else if constexpr (PH == 1) { p = make_float2(0.0f, J.re); q = make_float2(-J.im, 0.0f); }
    else if constexpr (PH == 2) { p = make_float2(J.im, 0.0f); q = make_float2(-J.re, 0.0f); }
    else { p = make_float2(0.0f, J.im); q = make_float2(J.re, 0.0f); }
    dot4_pairs(x, y, p, q);
    if constexpr (PH == 0) { J.re = p.x - p.y; J.im = q.x + q.y; }
    else if constexpr (PH == 1) { J.re = p.y - p.x; J.im = -(q.x + q.y); }
    else if constexpr (PH == 2) { J.im = p.x - p.y; J.re = -(q.x + q.y); }
    else { J.im = p.y - p.x; J.re = q.x + q.y; }
    return;
  }
  R tr, ti;  // the flow's parts that Re(XY) and Im(XY) add to, signed so both are +
  if constexpr (PH == 0) { tr = J.re; ti = J.im; }
  else if constexpr (PH == 1) { tr = -J.re; ti = -J.im; }
  else if constexpr (PH == 2) { tr = J.im; ti = -J.re; }   // J += i a: J.im += Re a, J.re -= Im a
  else { tr = -J.im; ti = J.re; }                          // J -= i a: J.im -= Re a, J.re += Im a
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    tr = fmac(x.w[k].re, y.w[k].re, tr);
    tr = fmac(-x.w[k].im, y.w[k].im, tr);
    ti = fmac(x.w[k].re, y.w[k].im, ti);
    ti = fmac(x.w[k].im, y.w[k].re, ti);
  }
  if constexpr (PH == 0) { J.re = tr; J.im = ti; }
  else if constexpr (PH == 1) { J.re = -tr; J.im = -ti; }
  else if constexpr (PH == 2) { J.im = tr; J.re = -ti; }
  else { J.im = -tr; J.re = ti; }
}

}  // namespace mg
