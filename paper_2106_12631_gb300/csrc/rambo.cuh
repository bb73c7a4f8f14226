// RAMBO for one event (Sec. 3: random numbers -> RAMBO -> momenta; Kleiss,
// Stirling, Ellis, CPC 40 (1986) 359), FP64, and its adjoint.
//
// Forward, per final-state particle i with uniforms r1..r4:
//   c = 2 r1 - 1, s = sqrt(1 - c^2), phi = 2 pi r2, e = -log(r3 r4)
//   q_i = e (1, s cos phi, s sin phi, c)
//   Q = sum q_i, M = sqrt(Q^2), b = -Qvec/M, g = Q0/M, a = 1/(1+g), x = ecm/M
//   p_i0 = x (g q_i0 + b.q_i),  p_i = x (q_i + b q_i0 + a (b.q_i) b)
// then, with masses, xi solves sum_i sqrt(m_i^2 + xi^2 p_i0^2) = ecm (Newton) and
//   k_i0 = sqrt(m_i^2 + xi^2 p_i0^2),  k_i = xi p_i.
// The adjoint reverses these steps; xi enters through the implicit-function
// derivative  d xi / d p_j0 = -(xi^2 p_j0 / k_j0) / sum_i (xi p_i0^2 / k_i0).
#pragma once
#include <cstdint>

namespace mg {

struct RamboSetup {
  double w0;       // flat massless volume (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!)
  int massive;     // any final-state mass != 0
  double xi0;      // Newton start sqrt(1 - (sum m / ecm)^2)
  double m2[4];    // final-state masses squared
};

template <int NF>
struct RamboState {
  double c[NF], s[NF], cp[NF], sp[NF], e[NF];
  double q[NF][4];
  double Q[4], M, b[3], g, a, x;
  double p[NF][4];   // massless momenta
  double xi;
  double k[NF][4];   // final momenta
  double w;
};

constexpr double kTwoPi = 6.283185307179586477;

// r: 4 NF uniforms of the event (r[4i + j])
template <int NF>
__device__ __forceinline__ void rambo_forward(const double* r, double ecm, const RamboSetup& st, RamboState<NF>& z) {
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    z.c[f] = 2.0 * r[4 * f] - 1.0;
    z.s[f] = sqrt(1.0 - z.c[f] * z.c[f]);
    sincos(kTwoPi * r[4 * f + 1], &z.sp[f], &z.cp[f]);
    z.e[f] = -log(r[4 * f + 2] * r[4 * f + 3]);
    z.q[f][0] = z.e[f];
    z.q[f][1] = z.e[f] * z.s[f] * z.cp[f];
    z.q[f][2] = z.e[f] * z.s[f] * z.sp[f];
    z.q[f][3] = z.e[f] * z.c[f];
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    z.Q[mu] = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) z.Q[mu] += z.q[f][mu];
  }
  z.M = sqrt(z.Q[0] * z.Q[0] - z.Q[1] * z.Q[1] - z.Q[2] * z.Q[2] - z.Q[3] * z.Q[3]);
  z.b[0] = -z.Q[1] / z.M; z.b[1] = -z.Q[2] / z.M; z.b[2] = -z.Q[3] / z.M;
  z.g = z.Q[0] / z.M;
  z.a = 1.0 / (1.0 + z.g);
  z.x = ecm / z.M;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double bq = z.b[0] * z.q[f][1] + z.b[1] * z.q[f][2] + z.b[2] * z.q[f][3];
    z.p[f][0] = z.x * (z.g * z.q[f][0] + bq);
#pragma unroll
    for (int k = 0; k < 3; ++k) z.p[f][k + 1] = z.x * (z.q[f][k + 1] + z.b[k] * z.q[f][0] + z.a * bq * z.b[k]);
  }
  z.w = st.w0;
  z.xi = 1.0;
  if (!st.massive) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) z.k[f][mu] = z.p[f][mu];
    return;
  }
  // Newton for sum_f sqrt(m_f^2 + xi^2 E_f^2) = ecm: first in FP32 to ~1e-6
  // (cheap; GB300 runs FP64 at 1/64 of the FP32 rate), then FP64 steps until
  // the residual is below 1e-15 ecm, plus one (quadratic convergence: the
  // same root as iterating in FP64 from the start)
  float xf = (float)st.xi0;
  for (int it = 0; it < 12; ++it) {
    float fv = -(float)ecm, df = 0.0f;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float e0 = (float)z.p[f][0];
      const float en = sqrtf((float)st.m2[f] + xf * xf * e0 * e0);
      fv += en;
      df += xf * e0 * e0 / en;
    }
    xf -= fv / df;
    if (fabsf(fv) <= 1e-6f * (float)ecm) break;
  }
  double xi = (isfinite(xf) && xf > 0.0f && xf <= 1.0f) ? (double)xf : st.xi0;  // else from the start
  int extra = 0;
  for (int it = 0; it < 50; ++it) {
    double fv = -ecm, df = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double en = sqrt(st.m2[f] + xi * xi * z.p[f][0] * z.p[f][0]);
      fv += en;
      df += xi * z.p[f][0] * z.p[f][0] / en;
    }
    xi -= fv / df;
    if (fabs(fv) <= 1e-15 * ecm && ++extra >= 1) break;
  }
  z.xi = xi;
  double w2 = 1.0, w3 = 0.0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double kk = xi * z.p[f][0];
    const double en = sqrt(st.m2[f] + kk * kk);
#pragma unroll
    for (int k = 1; k < 4; ++k) z.k[f][k] = xi * z.p[f][k];
    z.k[f][0] = en;
    w2 *= kk / en;
    w3 += kk * kk / en;
  }
  double pw = 1.0;
#pragma unroll
  for (int k = 0; k < 2 * NF - 3; ++k) pw *= xi;
  z.w = z.w * pw * w2 / w3 * ecm;
}

// kb[f][mu]: adjoint of the final momenta -> rb[4 f + j]: adjoint of the uniforms
template <int NF>
__device__ __forceinline__ void rambo_adjoint(const double* r, double ecm, const RamboSetup& st,
                                              const RamboState<NF>& z, const double (*kb)[4], double* rb) {
  double pb[NF][4];
  if (st.massive) {
    double xib = 0.0, fxi = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double p0 = z.p[f][0], k0 = z.k[f][0];
#pragma unroll
      for (int k = 1; k < 4; ++k) {
        pb[f][k] = z.xi * kb[f][k];
        xib += kb[f][k] * z.p[f][k];
      }
      xib += kb[f][0] * z.xi * p0 * p0 / k0;
      pb[f][0] = kb[f][0] * z.xi * z.xi * p0 / k0;
      fxi += z.xi * p0 * p0 / k0;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) pb[f][0] += xib * (-(z.xi * z.xi * z.p[f][0] / z.k[f][0]) / fxi);
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) pb[f][mu] = kb[f][mu];
  }
  // boost and scale back to the unconstrained q's
  double qb[NF][4];
  double xb = 0.0, gb = 0.0, ab = 0.0, bb[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double* q = z.q[f];
    const double bq = z.b[0] * q[1] + z.b[1] * q[2] + z.b[2] * q[3];
    double vb[3];
    xb += pb[f][0] * (z.g * q[0] + bq);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      xb += pb[f][k + 1] * (q[k + 1] + z.b[k] * q[0] + z.a * bq * z.b[k]);
      vb[k] = z.x * pb[f][k + 1];
    }
    const double P0 = z.x * pb[f][0];
    const double vbb = vb[0] * z.b[0] + vb[1] * z.b[1] + vb[2] * z.b[2];
    gb += P0 * q[0];
    qb[f][0] = P0 * z.g + vbb;
    const double bqb = P0 + z.a * vbb;
    ab += bq * vbb;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      qb[f][k + 1] = vb[k] + bqb * z.b[k];
      bb[k] += vb[k] * q[0] + z.a * bq * vb[k] + bqb * q[k + 1];
    }
  }
  gb += -ab * z.a * z.a;
  double Mb = -xb * z.x / z.M - gb * z.g / z.M;
  double Qb[4];
  Qb[0] = gb / z.M;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Qb[k + 1] = -bb[k] / z.M;
    Mb += -bb[k] * z.b[k] / z.M;
  }
  Qb[0] += Mb * z.Q[0] / z.M;
#pragma unroll
  for (int k = 1; k < 4; ++k) Qb[k] += -Mb * z.Q[k] / z.M;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) qb[f][mu] += Qb[mu];
    const double e = z.e[f], s = z.s[f], c = z.c[f], cp = z.cp[f], sp = z.sp[f];
    const double eb = qb[f][0] + qb[f][1] * s * cp + qb[f][2] * s * sp + qb[f][3] * c;
    const double sb = qb[f][1] * e * cp + qb[f][2] * e * sp;
    const double cb = qb[f][3] * e - sb * c / s;
    const double phib = -qb[f][1] * e * s * sp + qb[f][2] * e * s * cp;
    rb[4 * f + 0] = 2.0 * cb;
    rb[4 * f + 1] = kTwoPi * phib;
    rb[4 * f + 2] = -eb / r[4 * f + 2];
    rb[4 * f + 3] = -eb / r[4 * f + 3];
  }
}

}  // namespace mg
