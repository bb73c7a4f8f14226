// Complex numbers, wavefunction objects and couplings for the matrix-element
// kernels.  R is the working precision: double (plain FP64 path) or float
// (mixed path).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mg {

template <class R>
struct cx {
  R re, im;
  cx() = default;
  __host__ __device__ constexpr cx(R r, R i) : re(r), im(i) {}
};
template <class R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return cx<R>(a.re + b.re, a.im + b.im); }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return cx<R>(a.re - b.re, a.im - b.im); }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a) { return cx<R>(-a.re, -a.im); }
template <class R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return cx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return cx<R>(s * a.re, s * a.im); }
template <class R> __device__ __forceinline__ cx<R> operator*(cx<R> a, R s) { return cx<R>(s * a.re, s * a.im); }
template <class R> __device__ __forceinline__ cx<R>& operator+=(cx<R>& a, cx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> __device__ __forceinline__ cx<R>& operator-=(cx<R>& a, cx<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <class R> __device__ __forceinline__ cx<R> conj(cx<R> a) { return cx<R>(a.re, -a.im); }
template <class R> __device__ __forceinline__ cx<R> mul_i(cx<R> a) { return cx<R>(-a.im, a.re); }   // i * a
template <class R> __device__ __forceinline__ cx<R> mul_mi(cx<R> a) { return cx<R>(a.im, -a.re); }  // -i * a
// fused multiply-add in the working precision (one rounding)
template <class R> __device__ __forceinline__ R fmac(R a, R b, R c) {
  if constexpr (sizeof(R) == 4) return __fmaf_rn(a, b, c);
  else return __fma_rn(a, b, c);
}
// a b + c and s a + c as chains of fused multiply-adds (four and two
// operations; a product followed by a separate sum takes six and four)
template <class R> __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c) {
  return cx<R>(fmac(a.re, b.re, fmac(-a.im, b.im, c.re)), fmac(a.re, b.im, fmac(a.im, b.re, c.im)));
}
template <class R> __device__ __forceinline__ cx<R> rfma(R s, cx<R> a, cx<R> c) {
  return cx<R>(fmac(s, a.re, c.re), fmac(s, a.im, c.im));
}

// Four complex components: a Dirac spinor (chiral basis, upper pair
// left-handed; a row spinor for flowing-out fermions, a column spinor for
// flowing-in ones) or a Lorentz vector with upper index.  The paper's
// six-component wavefunction (Sec. 2) also carries the momentum; here the
// momenta are helicity independent and live in a per-event table instead.
template <class R>
struct alignas(16) W4 {
  cx<R> w[4];
};

// An array of N wavefunction slots stored as 16-byte planes: plane k holds
// bytes [16k, 16k + 16) of every slot.  Threads that read consecutive slots
// then touch consecutive 16-byte words of shared memory (no bank conflicts),
// and threads that read the same slot share one access.
template <class R, int N>
struct Slots {
  static constexpr int NPL = (int)(sizeof(W4<R>) / 16);
  uint4* p;
  __device__ __forceinline__ W4<R> operator[](int i) const {
    W4<R> w;
    uint4* d = reinterpret_cast<uint4*>(&w);
#pragma unroll
    for (int k = 0; k < NPL; ++k) d[k] = p[i + k * N];
    return w;
  }
  __device__ __forceinline__ void set(int i, const W4<R>& w) const {
    const uint4* s = reinterpret_cast<const uint4*>(&w);
#pragma unroll
    for (int k = 0; k < NPL; ++k) p[i + k * N] = s[k];
  }
  // slot i += w, component by component with shared-memory atomics (adjoint
  // accumulation from many threads)
  __device__ __forceinline__ void atomic_add(int i, const W4<R>& w) const {
    constexpr int PER = (int)(16 / sizeof(R));  // values per 16-byte plane word
    const R* s = reinterpret_cast<const R*>(&w);
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      R* d = reinterpret_cast<R*>(p + i + k * N);
#pragma unroll
      for (int q = 0; q < PER; ++q) atomicAdd(d + q, s[k * PER + q]);
    }
  }
};

// Couplings and masses in the working precision.
template <class R>
struct Couplings {
  R gs;    // strong coupling g_s (quark-gluon i g_s gamma^mu T^a, three-gluon g_s f^abc [..])
  R gs2;   // g_s^2 (four-gluon -i g_s^2 [..])
  R ee;    // e; photon-lepton vertex -i e Q gamma^mu with Q = -1
  R gz;    // e / (sin theta_W cos theta_W)
  R gzl;   // Z left coupling of charged leptons, T3 - Q sin^2 theta_W
  R gzr;   // Z right coupling, -Q sin^2 theta_W
  R mt;    // top mass
};

// Helicity-shared program tables (generated per process).
// One variant of one off-shell current or amputated current: type (0 ixxxxx,
// 1 oxxxxx, 2 vxxxxx, 3 off-shell flowing-out fermion, 4 off-shell flowing-in
// fermion, 5 vector from a fermion pair, 6 Z from a lepton pair, 7 three-gluon,
// 8 four-gluon term; amputated: 9 row, 10 column, 11 fermion pair, 12 lepton
// pair to Z, 13 three-gluon, 14 four-gluon term); a/b/c: type parameters
// (external: leg, helicity, flow sign; pair: coupling 0 g_s / 1 e); flag:
// external top mass; out/in: variant slots (a four-gluon term's three
// operands X_0, X_1, W); k0/k1: momentum-table entries; prop: propagator
// entry.  One aligned 16-byte word, read by one load.
struct alignas(16) HsItem {
  uint16_t out;
  uint16_t in[3];
  uint8_t type;
  int8_t a, b, c;
  uint8_t flag, k0, k1, prop;
};
static_assert(sizeof(HsItem) == 16, "item descriptor: one 16-byte word");
// Physics parameters in FP64 (propagator denominators are formed in FP64 in
// both precision modes).
struct PhysParams {
  double mz, wz, mt, wt;
};

}  // namespace mg
