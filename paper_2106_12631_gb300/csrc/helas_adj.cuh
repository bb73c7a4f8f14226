// Adjoints (reverse mode) of the helicity-amplitude routines in helas.cuh.
//
// Convention: for a real loss L and a complex intermediate z = x + i y the
// adjoint is zb = dL/dx + i dL/dy.  For w = f(z) holomorphic, zb += conj(f'(z)) wb;
// for a real input t entering a complex w, tb += Re(conj(dw/dt) wb).  Every
// routine below is multilinear in its wavefunction inputs, so its adjoint is
// the conjugate-transposed map, written out term by term from the forward
// formula (each comment names the forward routine).  Adjoint arguments are
// accumulated (+=).  Momentum adjoints Kb are real 4-vectors; propagator
// adjoints are complex.
#pragma once
#include <type_traits>

#include "helas.cuh"

namespace mg {

template <class R>
__device__ __forceinline__ W4<R> w4_zero() {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = cx<R>(R(0), R(0));
  return o;
}
template <class R>
__device__ __forceinline__ R re_dot(cx<R> a, cx<R> b) {  // Re(conj(a) b)
  return a.re * b.re + a.im * b.im;
}

// (vp, vm, xp, xm) = (V0 + V3, V0 - V3, V1 + i V2, V1 - i V2): scatter adjoints to V
template <class R>
__device__ __forceinline__ void slash_parts_adj(cx<R> bp, cx<R> bm, cx<R> bxp, cx<R> bxm, W4<R>& Vb) {
  Vb.w[0] += bp + bm;
  Vb.w[3] += bp - bm;
  Vb.w[1] += bxp + bxm;
  Vb.w[2] += mul_mi(bxp) + mul_i(bxm);
}

// row_slash: o0 = f2 vp + f3 xp, o1 = f2 xm + f3 vm, o2 = f0 vm - f1 xp, o3 = f1 vp - f0 xm
template <class R>
__device__ __forceinline__ void row_slash_adj(const W4<R>& f, const W4<R>& V, const W4<R>& ob, W4<R>& fb, W4<R>& Vb) {
  const cx<R> vp = V.w[0] + V.w[3], vm = V.w[0] - V.w[3];
  const cx<R> xp = V.w[1] + mul_i(V.w[2]), xm = V.w[1] - mul_i(V.w[2]);
  fb.w[2] += conj(vp) * ob.w[0] + conj(xm) * ob.w[1];
  fb.w[3] += conj(xp) * ob.w[0] + conj(vm) * ob.w[1];
  fb.w[0] += conj(vm) * ob.w[2] - conj(xm) * ob.w[3];
  fb.w[1] += conj(vp) * ob.w[3] - conj(xp) * ob.w[2];
  const cx<R> bp = conj(f.w[2]) * ob.w[0] + conj(f.w[1]) * ob.w[3];
  const cx<R> bm = conj(f.w[3]) * ob.w[1] + conj(f.w[0]) * ob.w[2];
  const cx<R> bxp = conj(f.w[3]) * ob.w[0] - conj(f.w[1]) * ob.w[2];
  const cx<R> bxm = conj(f.w[2]) * ob.w[1] - conj(f.w[0]) * ob.w[3];
  slash_parts_adj(bp, bm, bxp, bxm, Vb);
}

// row_kslash_m: o0 = kp f2 + f3 kxp + m f0, o1 = f2 kxm + km f3 + m f1,
//               o2 = km f0 - f1 kxp + m f2, o3 = kp f1 - f0 kxm + m f3
template <class R>
__device__ __forceinline__ void row_kslash_m_adj(const W4<R>& f, const R* K, R m, const W4<R>& ob, W4<R>& fb, R* Kb) {
  const R kp = K[0] + K[3], km = K[0] - K[3];
  const cx<R> kxp(K[1], K[2]), kxm(K[1], -K[2]);
  fb.w[0] += m * ob.w[0] + km * ob.w[2] - conj(kxm) * ob.w[3];
  fb.w[1] += m * ob.w[1] - conj(kxp) * ob.w[2] + kp * ob.w[3];
  fb.w[2] += kp * ob.w[0] + conj(kxm) * ob.w[1] + m * ob.w[2];
  fb.w[3] += conj(kxp) * ob.w[0] + km * ob.w[1] + m * ob.w[3];
  const R bkp = re_dot(f.w[2], ob.w[0]) + re_dot(f.w[1], ob.w[3]);
  const R bkm = re_dot(f.w[3], ob.w[1]) + re_dot(f.w[0], ob.w[2]);
  const cx<R> bxp = conj(f.w[3]) * ob.w[0] - conj(f.w[1]) * ob.w[2];
  const cx<R> bxm = conj(f.w[2]) * ob.w[1] - conj(f.w[0]) * ob.w[3];
  Kb[0] += bkp + bkm;
  Kb[3] += bkp - bkm;
  Kb[1] += bxp.re + bxm.re;
  Kb[2] += bxp.im - bxm.im;
}

// FFV1_0 = i g row_col(row_slash(fo, v), fi)
template <class R>
__device__ __forceinline__ void FFV1_0_adj(const W4<R>& fo, const W4<R>& fi, const W4<R>& v, R g, cx<R> ab, W4<R>& fob,
                                           W4<R>& fib, W4<R>& vb) {
  const W4<R> r = row_slash(fo, v);
  const cx<R> sb = mul_mi(g * ab);  // conj(i g) ab
  W4<R> rb;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    rb.w[k] = conj(fi.w[k]) * sb;
    fib.w[k] += conj(r.w[k]) * sb;
  }
  row_slash_adj(fo, v, rb, fob, vb);
}

// FFV1_2 = [row_kslash_m(row_slash(fo, v), K, m)] (i g prop)
template <class R>
__device__ __forceinline__ void FFV1_2_adj(const W4<R>& fo, const W4<R>& v, R g, const R* K, R m, cx<R> prop,
                                           const W4<R>& ob, W4<R>& fob, W4<R>& vb, R* Kb, cx<R>& propb) {
  const W4<R> u = row_slash(fo, v);
  const W4<R> w = row_kslash_m(u, K, m);
  const cx<R> s = mul_i(g * prop);
  W4<R> wb;
  cx<R> sb(R(0), R(0));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wb.w[k] = conj(s) * ob.w[k];
    sb += conj(w.w[k]) * ob.w[k];
  }
  propb += mul_mi(g * sb);  // conj(i g) sb
  W4<R> ub = w4_zero<R>();
  row_kslash_m_adj(u, K, m, wb, ub, Kb);
  row_slash_adj(fo, v, ub, fob, vb);
}

// VVV1P0_1 = (d12 (a1.a2) + a2 (d23.a1) + a1 (d31.a2)) g prop,
// d12 = K2 - K1, d23 = -(K1 + 2 K2), d31 = 2 K1 + K2
template <class R>
__device__ __forceinline__ void VVV1P0_1_adj(const W4<R>& a1, const W4<R>& a2, const R* K1, const R* K2, R g, cx<R> prop,
                                             const W4<R>& ob, W4<R>& a1b, W4<R>& a2b, R* K1b, R* K2b, cx<R>& propb) {
  R d12[4], d23[4], d31[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    d12[mu] = K2[mu] - K1[mu];
    d23[mu] = -(K1[mu] + R(2) * K2[mu]);
    d31[mu] = R(2) * K1[mu] + K2[mu];
  }
  const cx<R> a12 = vdot(a1, a2), c1 = kdot(d23, a1), c2 = kdot(d31, a2);
  const cx<R> s = g * prop;
  cx<R> sb(R(0), R(0)), a12b(R(0), R(0)), c1b(R(0), R(0)), c2b(R(0), R(0));
  R d12b[4], d23b[4], d31b[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const cx<R> t = d12[mu] * a12 + a2.w[mu] * c1 + a1.w[mu] * c2;
    const cx<R> tb = conj(s) * ob.w[mu];
    sb += conj(t) * ob.w[mu];
    a12b += d12[mu] * tb;
    d12b[mu] = re_dot(a12, tb);
    a2b.w[mu] += conj(c1) * tb;
    c1b += conj(a2.w[mu]) * tb;
    a1b.w[mu] += conj(c2) * tb;
    c2b += conj(a1.w[mu]) * tb;
  }
  propb += g * sb;
  const R eta[4] = {R(1), R(-1), R(-1), R(-1)};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    a1b.w[mu] += (eta[mu] * d23[mu]) * c1b + eta[mu] * (conj(a2.w[mu]) * a12b);
    a2b.w[mu] += (eta[mu] * d31[mu]) * c2b + eta[mu] * (conj(a1.w[mu]) * a12b);
    d23b[mu] = eta[mu] * re_dot(a1.w[mu], c1b);
    d31b[mu] = eta[mu] * re_dot(a2.w[mu], c2b);
    K1b[mu] += -d12b[mu] - d23b[mu] + R(2) * d31b[mu];
    K2b[mu] += d12b[mu] - R(2) * d23b[mu] + d31b[mu];
  }
}

// four-gluon terms: o = ((A.B) X - (C.D) Y) (-i g2 prop)
template <class R>
__device__ __forceinline__ void vvvv_adj(const W4<R>& X, const W4<R>& A, const W4<R>& B, const W4<R>& Y, const W4<R>& C,
                                         const W4<R>& D, R g2, cx<R> prop, const W4<R>& ob, W4<R>& Xb, W4<R>& Ab,
                                         W4<R>& Bb, W4<R>& Yb, W4<R>& Cb, W4<R>& Db, cx<R>& propb) {
  const cx<R> cxv = vdot(A, B), cyv = vdot(C, D);
  const cx<R> s = mul_mi(g2 * prop);
  cx<R> sb(R(0), R(0)), cxb(R(0), R(0)), cyb(R(0), R(0));
  W4<R> tb;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const cx<R> t = cxv * X.w[mu] - cyv * Y.w[mu];
    tb.w[mu] = conj(s) * ob.w[mu];
    sb += conj(t) * ob.w[mu];
    cxb += conj(X.w[mu]) * tb.w[mu];
    cyb -= conj(Y.w[mu]) * tb.w[mu];
  }
  propb += mul_i(g2 * sb);  // conj(-i g2) sb
  const R eta[4] = {R(1), R(-1), R(-1), R(-1)};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    Xb.w[mu] += conj(cxv) * tb.w[mu];
    Yb.w[mu] -= conj(cyv) * tb.w[mu];
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    Ab.w[mu] += eta[mu] * (conj(B.w[mu]) * cxb);
    Bb.w[mu] += eta[mu] * (conj(A.w[mu]) * cxb);
    Cb.w[mu] += eta[mu] * (conj(D.w[mu]) * cyb);
    Db.w[mu] += eta[mu] * (conj(C.w[mu]) * cyb);
  }
}
// VVVV1P0_1: (a1.a3) a2 - (a2.a3) a1
template <class R>
__device__ __forceinline__ void VVVV1P0_1_adj(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, R g2, cx<R> prop,
                                              const W4<R>& ob, W4<R>& a1b, W4<R>& a2b, W4<R>& a3b, cx<R>& propb) {
  vvvv_adj(a2, a1, a3, a1, a2, a3, g2, prop, ob, a2b, a1b, a3b, a1b, a2b, a3b, propb);
}
// VVVV3P0_1: (a1.a2) a3 - (a2.a3) a1
template <class R>
__device__ __forceinline__ void VVVV3P0_1_adj(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, R g2, cx<R> prop,
                                              const W4<R>& ob, W4<R>& a1b, W4<R>& a2b, W4<R>& a3b, cx<R>& propb) {
  vvvv_adj(a3, a1, a2, a1, a2, a3, g2, prop, ob, a3b, a1b, a2b, a1b, a2b, a3b, propb);
}
// VVVV4P0_1: (a1.a2) a3 - (a1.a3) a2
template <class R>
__device__ __forceinline__ void VVVV4P0_1_adj(const W4<R>& a1, const W4<R>& a2, const W4<R>& a3, R g2, cx<R> prop,
                                              const W4<R>& ob, W4<R>& a1b, W4<R>& a2b, W4<R>& a3b, cx<R>& propb) {
  vvvv_adj(a3, a1, a2, a2, a1, a3, g2, prop, ob, a3b, a1b, a2b, a2b, a1b, a3b, propb);
}

// slash_col: o0 = vm f2 - xm f3, o1 = vp f3 - xp f2, o2 = vp f0 + xm f1, o3 = xp f0 + vm f1
template <class R>
__device__ __forceinline__ void slash_col_adj(const W4<R>& V, const W4<R>& f, const W4<R>& ob, W4<R>& Vb, W4<R>& fb) {
  const cx<R> vp = V.w[0] + V.w[3], vm = V.w[0] - V.w[3];
  const cx<R> xp = V.w[1] + mul_i(V.w[2]), xm = V.w[1] - mul_i(V.w[2]);
  fb.w[2] += conj(vm) * ob.w[0] - conj(xp) * ob.w[1];
  fb.w[3] += conj(vp) * ob.w[1] - conj(xm) * ob.w[0];
  fb.w[0] += conj(vp) * ob.w[2] + conj(xp) * ob.w[3];
  fb.w[1] += conj(xm) * ob.w[2] + conj(vm) * ob.w[3];
  const cx<R> bp = conj(f.w[3]) * ob.w[1] + conj(f.w[0]) * ob.w[2];
  const cx<R> bm = conj(f.w[2]) * ob.w[0] + conj(f.w[1]) * ob.w[3];
  const cx<R> bxp = conj(f.w[0]) * ob.w[3] - conj(f.w[2]) * ob.w[1];
  const cx<R> bxm = conj(f.w[1]) * ob.w[2] - conj(f.w[3]) * ob.w[0];
  slash_parts_adj(bp, bm, bxp, bxm, Vb);
}

// mkslash_m_col: o0 = m f0 - (km f2 - kxm f3), o1 = m f1 - (kp f3 - kxp f2),
//                o2 = m f2 - (kp f0 + kxm f1), o3 = m f3 - (kxp f0 + km f1)
template <class R>
__device__ __forceinline__ void mkslash_m_col_adj(const R* K, R m, const W4<R>& f, const W4<R>& ob, W4<R>& fb, R* Kb) {
  const R kp = K[0] + K[3], km = K[0] - K[3];
  const cx<R> kxp(K[1], K[2]), kxm(K[1], -K[2]);
  fb.w[0] += m * ob.w[0] - kp * ob.w[2] - conj(kxp) * ob.w[3];
  fb.w[1] += m * ob.w[1] - conj(kxm) * ob.w[2] - km * ob.w[3];
  fb.w[2] += m * ob.w[2] - km * ob.w[0] + conj(kxp) * ob.w[1];
  fb.w[3] += m * ob.w[3] + conj(kxm) * ob.w[0] - kp * ob.w[1];
  const R bkp = -re_dot(f.w[3], ob.w[1]) - re_dot(f.w[0], ob.w[2]);
  const R bkm = -re_dot(f.w[2], ob.w[0]) - re_dot(f.w[1], ob.w[3]);
  Kb[0] += bkp + bkm;
  Kb[3] += bkp - bkm;
  // d o / d K1: o0 += f3, o1 += f2, o2 -= f1, o3 -= f0; d o / d K2: i times (-f3, f2, f1, -f0)
  Kb[1] += re_dot(f.w[3], ob.w[0]) + re_dot(f.w[2], ob.w[1]) - re_dot(f.w[1], ob.w[2]) - re_dot(f.w[0], ob.w[3]);
  Kb[2] += re_dot(mul_mi(f.w[3]), ob.w[0]) + re_dot(mul_i(f.w[2]), ob.w[1]) + re_dot(mul_i(f.w[1]), ob.w[2]) +
           re_dot(mul_mi(f.w[0]), ob.w[3]);
}

// FFV1_1 = [mkslash_m_col(K, m, slash_col(v, fi))] (i g prop)
template <class R>
__device__ __forceinline__ void FFV1_1_adj(const W4<R>& fi, const W4<R>& v, R g, const R* K, R m, cx<R> prop,
                                           const W4<R>& ob, W4<R>& fib, W4<R>& vb, R* Kb, cx<R>& propb) {
  const W4<R> u = slash_col(v, fi);
  const W4<R> w = mkslash_m_col(K, m, u);
  const cx<R> s = mul_i(g * prop);
  W4<R> wb;
  cx<R> sb(R(0), R(0));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wb.w[k] = conj(s) * ob.w[k];
    sb += conj(w.w[k]) * ob.w[k];
  }
  propb += mul_mi(g * sb);
  W4<R> ub = w4_zero<R>();
  mkslash_m_col_adj(K, m, u, wb, ub, Kb);
  slash_col_adj(v, fi, ub, vb, fib);
}

// bilinear (row f, column g, couplings gl, gr): see helas.cuh
template <class R>
__device__ __forceinline__ void bilinear_adj(const W4<R>& f, const W4<R>& g, R gl, R gr, const W4<R>& jb, W4<R>& fb,
                                             W4<R>& gb) {
  const cx<R> a02b = gr * (jb.w[0] + jb.w[3]), a13b = gr * (jb.w[0] - jb.w[3]);
  const cx<R> a03b = gr * (jb.w[1] + mul_i(jb.w[2])), a12b = gr * (jb.w[1] - mul_i(jb.w[2]));
  const cx<R> b20b = gl * (jb.w[0] - jb.w[3]), b31b = gl * (jb.w[0] + jb.w[3]);
  const cx<R> b21b = gl * (-jb.w[1] - mul_i(jb.w[2])), b30b = gl * (mul_i(jb.w[2]) - jb.w[1]);
  fb.w[0] += conj(g.w[2]) * a02b + conj(g.w[3]) * a03b;
  fb.w[1] += conj(g.w[3]) * a13b + conj(g.w[2]) * a12b;
  fb.w[2] += conj(g.w[0]) * b20b + conj(g.w[1]) * b21b;
  fb.w[3] += conj(g.w[1]) * b31b + conj(g.w[0]) * b30b;
  gb.w[2] += conj(f.w[0]) * a02b + conj(f.w[1]) * a12b;
  gb.w[3] += conj(f.w[1]) * a13b + conj(f.w[0]) * a03b;
  gb.w[0] += conj(f.w[2]) * b20b + conj(f.w[3]) * b30b;
  gb.w[1] += conj(f.w[3]) * b31b + conj(f.w[2]) * b21b;
}

// FFV1P0_3 = bilinear(fo, fi, 1, 1) (i g prop)
template <class R>
__device__ __forceinline__ void FFV1P0_3_adj(const W4<R>& fo, const W4<R>& fi, R g, cx<R> prop, const W4<R>& ob,
                                             W4<R>& fob, W4<R>& fib, cx<R>& propb) {
  const W4<R> j = bilinear(fo, fi, R(1), R(1));
  const cx<R> s = mul_i(g * prop);
  W4<R> jb;
  cx<R> sb(R(0), R(0));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    jb.w[k] = conj(s) * ob.w[k];
    sb += conj(j.w[k]) * ob.w[k];
  }
  propb += mul_mi(g * sb);
  bilinear_adj(fo, fi, R(1), R(1), jb, fob, fib);
}

// ---- amputated currents (helas.cuh): same maps without the propagator,
// vector outputs with a lower index (o_mu = eta_mu t_mu)
template <class R>
__device__ __forceinline__ W4<R> lower_adj(const W4<R>& ob) {  // adjoint seen by the upper-index vector
  W4<R> t;
  t.w[0] = ob.w[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) t.w[k] = -ob.w[k];
  return t;
}
// FFV1_2A = i g row_slash(fo, v)
template <class R>
__device__ __forceinline__ void FFV1_2A_adj(const W4<R>& fo, const W4<R>& v, R g, const W4<R>& ob, W4<R>& fob,
                                            W4<R>& vb) {
  W4<R> ub;
#pragma unroll
  for (int k = 0; k < 4; ++k) ub.w[k] = mul_mi(g * ob.w[k]);
  row_slash_adj(fo, v, ub, fob, vb);
}
// FFV1_1A = i g slash_col(v, fi)
template <class R>
__device__ __forceinline__ void FFV1_1A_adj(const W4<R>& fi, const W4<R>& v, R g, const W4<R>& ob, W4<R>& fib,
                                            W4<R>& vb) {
  W4<R> ub;
#pragma unroll
  for (int k = 0; k < 4; ++k) ub.w[k] = mul_mi(g * ob.w[k]);
  slash_col_adj(v, fi, ub, vb, fib);
}
// FFV1P0_3A = lower(i g bilinear(fo, fi, 1, 1))
template <class R>
__device__ __forceinline__ void FFV1P0_3A_adj(const W4<R>& fo, const W4<R>& fi, R g, const W4<R>& ob, W4<R>& fob,
                                              W4<R>& fib) {
  const W4<R> t = lower_adj(ob);
  W4<R> jb;
#pragma unroll
  for (int k = 0; k < 4; ++k) jb.w[k] = mul_mi(g * t.w[k]);
  bilinear_adj(fo, fi, R(1), R(1), jb, fob, fib);
}
// VVV1P0_1A = lower(g n): VVV1P0_1 with a unit propagator
template <class R>
__device__ __forceinline__ void VVV1P0_1A_adj(const W4<R>& a1, const W4<R>& a2, const R* K1, const R* K2, R g,
                                              const W4<R>& ob, W4<R>& a1b, W4<R>& a2b, R* K1b, R* K2b) {
  cx<R> unused(R(0), R(0));
  VVV1P0_1_adj(a1, a2, K1, K2, g, cx<R>(R(1), R(0)), lower_adj(ob), a1b, a2b, K1b, K2b, unused);
}
// vvvv_comb_a = lower(-i g2 ((A.B) X - (C.D) Y)): vvvv_adj with a unit propagator
template <class R>
__device__ __forceinline__ void vvvv_comb_a_adj(const W4<R>& X, const W4<R>& A, const W4<R>& B, const W4<R>& Y,
                                                const W4<R>& C, const W4<R>& D, R g2, const W4<R>& ob, W4<R>& Xb,
                                                W4<R>& Ab, W4<R>& Bb, W4<R>& Yb, W4<R>& Cb, W4<R>& Db) {
  cx<R> unused(R(0), R(0));
  vvvv_adj(X, A, B, Y, C, D, g2, cx<R>(R(1), R(0)), lower_adj(ob), Xb, Ab, Bb, Yb, Cb, Db, unused);
}

// contraction A = sum_i X_i Y_i: Xb_i += conj(Y_i) Ab (and symmetrically)
template <class R>
__device__ __forceinline__ void w4_acc_conj(W4<R>& acc, const W4<R>& y, cx<R> ab) {
#pragma unroll
  for (int k = 0; k < 4; ++k) acc.w[k] += conj(y.w[k]) * ab;
}
template <class R>
__device__ __forceinline__ W4<R> w4_conj_scale(const W4<R>& x, cx<R> ab) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = conj(x.w[k]) * ab;
  return o;
}
// sum of v over the lanes that differ only in the lane bits of MASK (butterfly);
// every lane of the warp must take part
template <unsigned MASK, class R>
__device__ __forceinline__ void w4_warp_sum(W4<R>& v) {
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if (!(MASK >> b & 1u)) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v.w[k].re += __shfl_xor_sync(0xffffffffu, v.w[k].re, 1 << b);
      v.w[k].im += __shfl_xor_sync(0xffffffffu, v.w[k].im, 1 << b);
    }
  }
}

// y times i, -1, -i
template <class R>
__device__ __forceinline__ W4<R> w4_mul_i(const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = mul_i(y.w[k]);
  return o;
}
template <class R>
__device__ __forceinline__ W4<R> w4_neg(const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = -y.w[k];
  return o;
}
template <class R>
__device__ __forceinline__ W4<R> w4_mul_mi(const W4<R>& y) {
  W4<R> o;
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] = mul_mi(y.w[k]);
  return o;
}

// Propagator factor prop = c / (K^2 - M^2 + i M W), c = i (fermion) or -i (vector):
// d prop / d K_mu = kappa 2 eta_mu K_mu with kappa = i prop^2 (fermion), -i prop^2 (vector)
template <class R>
__device__ __forceinline__ void prop_adj(cx<R> prop, bool fermion, const R* K, cx<R> propb, R* Kb) {
  const cx<R> p2 = prop * prop;
  const cx<R> kappa = fermion ? mul_i(p2) : mul_mi(p2);
  const R f = R(2) * re_dot(kappa, propb);
  Kb[0] += f * K[0];
  Kb[1] -= f * K[1];
  Kb[2] -= f * K[2];
  Kb[3] -= f * K[3];
}

// ---- external wavefunctions: momentum Jacobian by forward mode ----------------
// A number with derivatives along the four momentum components.
template <class R>
struct D4 {
  R v, d[4];
  D4() = default;
  template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
  __device__ __forceinline__ D4(T x) : v(R(x)) {
    d[0] = d[1] = d[2] = d[3] = R(0);
  }
};
using ::sqrt;
template <class R> __device__ __forceinline__ D4<R> operator+(D4<R> a, D4<R> b) { D4<R> r(a.v + b.v); for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <class R> __device__ __forceinline__ D4<R> operator-(D4<R> a, D4<R> b) { D4<R> r(a.v - b.v); for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <class R> __device__ __forceinline__ D4<R> operator-(D4<R> a) { D4<R> r(-a.v); for (int k = 0; k < 4; ++k) r.d[k] = -a.d[k]; return r; }
template <class R> __device__ __forceinline__ D4<R> operator*(D4<R> a, D4<R> b) { D4<R> r(a.v * b.v); for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <class R> __device__ __forceinline__ D4<R> operator/(D4<R> a, D4<R> b) {
  D4<R> r(a.v / b.v);
  const R ib = R(1) / b.v;
  for (int k = 0; k < 4; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <class R> __device__ __forceinline__ D4<R>& operator+=(D4<R>& a, D4<R> b) { a = a + b; return a; }
template <class R> __device__ __forceinline__ D4<R>& operator-=(D4<R>& a, D4<R> b) { a = a - b; return a; }
template <class R> __device__ __forceinline__ bool operator>=(D4<R> a, D4<R> b) { return a.v >= b.v; }
template <class R> __device__ __forceinline__ bool operator<=(D4<R> a, D4<R> b) { return a.v <= b.v; }
template <class R> __device__ __forceinline__ bool operator==(D4<R> a, D4<R> b) { return a.v == b.v; }
template <class R> __device__ __forceinline__ D4<R> sqrt(D4<R> a) {
  D4<R> r(sqrt(a.v));
  const R h = R(0.5) / r.v;
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <> __device__ __forceinline__ D4<float> rsqrt_<D4<float>>(D4<float> x) { return D4<float>(1.0f) / sqrt(x); }
template <> __device__ __forceinline__ D4<double> rsqrt_<D4<double>>(D4<double> x) { return D4<double>(1.0) / sqrt(x); }

// pb_nu += Re(sum_c conj(dW_c/dp_nu) Wb_c) for an external wavefunction W(p).
// kind: 0 ixxxxx, 1 oxxxxx, 2 vxxxxx.
template <class R>
__device__ __forceinline__ void external_adj(int kind, const R* p, R m, int hel, int ns, const W4<R>& wb, R* pb) {
  D4<R> pd[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) { pd[mu] = D4<R>(p[mu]); pd[mu].d[mu] = R(1); }
  W4<D4<R>> w;
  if (kind == 0) w = ixxxxx<D4<R>>(pd, D4<R>(m), hel, ns);
  else if (kind == 1) w = oxxxxx<D4<R>>(pd, D4<R>(m), hel, ns);
  else w = vxxxxx<D4<R>>(pd, hel, ns);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) pb[nu] += w.w[c].re.d[nu] * wb.w[c].re + w.w[c].im.d[nu] * wb.w[c].im;
}

// slot i += w by its only writer (a plain read, add and write: the adjoint
// contractions' warp sums leave one lane per slot and event)
// ---- sum of a W4 over a group of lanes, added into a slot -----------------
// The lanes that differ only in the bits of MASK (at most the five lane bits)
// hold terms of one slot's adjoint.  Reduce-scatter: at each of the first
// (up to three) bits of MASK the two partner lanes swap half of the
// components they still hold and each keeps the sum of the other half (4, 2,
// then 1 values exchanged instead of all 8 per level); further bits sum the
// kept components; every lane whose further bits are 0 then adds its
// components into the slot (each component has one writing lane).
constexpr int popc5(unsigned m) {
  return (int)(m & 1u) + (int)(m >> 1 & 1u) + (int)(m >> 2 & 1u) + (int)(m >> 3 & 1u) + (int)(m >> 4 & 1u);
}
constexpr int nth_set_bit(unsigned m, int t) {
  for (int b = 0; b < 32; ++b)
    if (m >> b & 1u) {
      if (t == 0) return b;
      --t;
    }
  return -1;
}
constexpr unsigned drop_low_set_bits(unsigned m, int k) {
  for (int i = 0; i < k; ++i) m &= m - 1u;
  return m;
}

template <unsigned MASK, int T, int S, class R>
__device__ __forceinline__ void rs_split(R* v, int lane, int& off) {
  if constexpr (T < S) {
    constexpr int b = nth_set_bit(MASK, T), h = (8 >> T) / 2;
    const bool hi = (lane >> b & 1) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const R send = hi ? v[j] : v[h + j];
      const R keep = hi ? v[h + j] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << b);
    }
    off += hi ? h : 0;
    rs_split<MASK, T + 1, S, R>(v, lane, off);
  }
}

template <unsigned MASK, int T, int NB, int K, class R>
__device__ __forceinline__ void rs_sum(R* v) {
  if constexpr (T < NB) {
    constexpr int b = nth_set_bit(MASK, T);
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 1 << b);
    rs_sum<MASK, T + 1, NB, K, R>(v);
  }
}

// ATOMIC: the slot also receives adds from other warps (shared-memory atomics).
template <unsigned MASK, bool ATOMIC, class R, int N>
__device__ __forceinline__ void w4_warp_reduce_add(const W4<R>& w, const Slots<R, N>& s, int i, int lane, bool act) {
  static_assert(MASK < 32u, "lane bits only");
  constexpr int NB = popc5(MASK), S = NB < 3 ? NB : 3, K = 8 >> S;
  R v[8] = {w.w[0].re, w.w[0].im, w.w[1].re, w.w[1].im, w.w[2].re, w.w[2].im, w.w[3].re, w.w[3].im};
  int off = 0;  // first of the K components this lane keeps
  rs_split<MASK, 0, S, R>(v, lane, off);
  rs_sum<MASK, S, NB, K, R>(v);
  constexpr unsigned REST = drop_low_set_bits(MASK, S);
  if ((lane & (int)REST) == 0 && act) {
    constexpr int PER = (int)(16 / sizeof(R));  // components per 16-byte plane
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int c = off + j;
      R* d = reinterpret_cast<R*>(s.p + i + (c / PER) * N) + (c % PER);
      if constexpr (ATOMIC) atomicAdd(d, v[j]);
      else *d += v[j];
    }
  }
}

template <class R, int N>
__device__ __forceinline__ void slot_add(const Slots<R, N>& s, int i, const W4<R>& w) {
  W4<R> o = s[i];
#pragma unroll
  for (int k = 0; k < 4; ++k) o.w[k] += w.w[k];
  s.set(i, o);
}

}  // namespace mg
