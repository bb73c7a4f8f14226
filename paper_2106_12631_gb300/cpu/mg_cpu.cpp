// SIMD CPU build of the helicity-shared matrix-element program (Sec. 4: the
// C++ build of the same event-parallel code, the innermost loop over the
// contiguous events of one vector, several events per SIMD instruction).
//
// The wavefunction, current, amputated-current and contraction routines are
// the GPU path's own (helas.cuh and the generated process programs), compiled
// here for the host with a "lane" type in place of the scalar: one Lane holds
// the same quantity for MGC_LANES_BYTES / sizeof(T) events and every
// arithmetic operator acts on all of them (GCC vector extensions: 128-bit NEON
// on Grace, SSE2 on x86-64, no target-specific flags).  The external
// wavefunctions (which branch on the momenta), the momentum sums and the
// propagator denominators are formed per event in FP64 and packed into lanes.
// Per block of lanes: externals and tables, the current variants level by
// level, then chunk by chunk the amputated currents and, for every good
// helicity, the contractions into its colour flows; the colour sum J^dagger C J
// per helicity in the lane precision and the helicity sum in FP64 per event.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include <cuda_runtime.h>  // the vector structs (float2, uint4) the shared headers use

// Host stand-ins for the device intrinsics the shared headers name.
static inline void __syncthreads() {}
static inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
  return make_float2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
}
static inline float2 __fmul2_rn(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
static inline float2 __fadd2_rn(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

#include "mg_cpu.h"
#include "process.cuh"

#ifndef MGC_LANES_BYTES
#define MGC_LANES_BYTES 64  // bytes per lane vector: 16 FP32 or 8 FP64 events (wider ran faster on Grace but compiles for minutes)
#endif

namespace mgcpu {

template <class T, int W>
struct Lane {
  typedef T vec __attribute__((vector_size(W * sizeof(T))));
  vec v;
  Lane() = default;
  Lane(double s) {
    for (int i = 0; i < W; ++i) v[i] = (T)s;
  }
  static Lane of(vec x) {
    Lane l;
    l.v = x;
    return l;
  }
};
template <class T, int W> inline Lane<T, W> operator+(Lane<T, W> a, Lane<T, W> b) { return Lane<T, W>::of(a.v + b.v); }
template <class T, int W> inline Lane<T, W> operator-(Lane<T, W> a, Lane<T, W> b) { return Lane<T, W>::of(a.v - b.v); }
template <class T, int W> inline Lane<T, W> operator*(Lane<T, W> a, Lane<T, W> b) { return Lane<T, W>::of(a.v * b.v); }
template <class T, int W> inline Lane<T, W> operator/(Lane<T, W> a, Lane<T, W> b) { return Lane<T, W>::of(a.v / b.v); }
template <class T, int W> inline Lane<T, W> operator-(Lane<T, W> a) { return Lane<T, W>::of(-a.v); }
template <class T, int W> inline Lane<T, W>& operator+=(Lane<T, W>& a, Lane<T, W> b) { a.v += b.v; return a; }
template <class T, int W> inline Lane<T, W>& operator-=(Lane<T, W>& a, Lane<T, W> b) { a.v -= b.v; return a; }
// the shared headers' fused multiply-add, lane by lane (found by argument-
// dependent lookup; the compiler contracts it to vector FMAs where the target has them)
template <class T, int W> inline Lane<T, W> fmac(Lane<T, W> a, Lane<T, W> b, Lane<T, W> c) {
  return Lane<T, W>::of(a.v * b.v + c.v);
}

template <class R>
struct SlotArray {  // the current / amputated-current slots of one block
  mg::W4<R>* p;
  mg::W4<R> operator[](int i) const { return p[i]; }
};

template <class P>
mg::W4<double> external(const mg::HsItem& it, const double* k, double mt) {
  if (it.type == 0) return mg::ixxxxx<double>(k, it.flag ? mt : 0.0, it.b, it.c);
  if (it.type == 1) return mg::oxxxxx<double>(k, it.flag ? mt : 0.0, it.b, it.c);
  return mg::vxxxxx<double>(k, it.b, it.c);
}

// one current variant (as the GPU's hs_item, on lanes)
template <class P, class R>
inline void item(const mg::HsItem& it, mg::W4<R>* cur, const R* K, const mg::cx<R>* pr, const mg::Couplings<R>& cp) {
  using namespace mg;
  W4<R> o;
  switch (it.type) {
    case 3: o = FFV1_2<R>(cur[it.in[0]], cur[it.in[1]], cp.gs, K + 4 * it.k0, cp.mt, pr[it.prop]); break;
    case 4: o = FFV1_1<R>(cur[it.in[0]], cur[it.in[1]], cp.gs, K + 4 * it.k0, cp.mt, pr[it.prop]); break;
    case 5: o = FFV1P0_3<R>(cur[it.in[0]], cur[it.in[1]], it.a ? cp.ee : cp.gs, pr[it.prop]); break;
    case 6: o = FFV2_4_3<R>(cur[it.in[0]], cur[it.in[1]], cp.gz, cp.gzl, cp.gzr, pr[it.prop]); break;
    case 7: o = VVV1P0_1<R>(cur[it.in[0]], cur[it.in[1]], K + 4 * it.k0, K + 4 * it.k1, cp.gs, pr[it.prop]); break;
    default:  // four-gluon term X_0 (X_1 . W) - X_1 (X_0 . W), in = {X_0, X_1, W}
      o = vvvv_comb(cur[it.in[0]], vdot(cur[it.in[1]], cur[it.in[2]]), cur[it.in[1]],
                    vdot(cur[it.in[0]], cur[it.in[2]]), mul_mi(cp.gs2 * pr[it.prop]));
  }
  cur[it.out] = o;
}

// one amputated-current variant (as the GPU's hs_xitem)
template <class P, class R>
inline void xitem(const mg::HsItem& it, const mg::W4<R>* cur, mg::W4<R>* xb, const R* K, const mg::Couplings<R>& cp) {
  using namespace mg;
  W4<R> o;
  switch (it.type) {
    case 9: o = FFV1_2A<R>(cur[it.in[0]], cur[it.in[1]], cp.gs); break;
    case 10: o = FFV1_1A<R>(cur[it.in[0]], cur[it.in[1]], cp.gs); break;
    case 11: o = FFV1P0_3A<R>(cur[it.in[0]], cur[it.in[1]], it.a ? cp.ee : cp.gs); break;
    case 12: o = FFV2_4_3A<R>(cur[it.in[0]], cur[it.in[1]], cp.gz, cp.gzl, cp.gzr); break;
    case 13: o = VVV1P0_1A<R>(cur[it.in[0]], cur[it.in[1]], K + 4 * it.k0, K + 4 * it.k1, cp.gs); break;
    default:  // four-gluon term, as in item
      o = vvvv_comb_a(cur[it.in[0]], vdot(cur[it.in[1]], cur[it.in[2]]), cur[it.in[1]],
                      vdot(cur[it.in[0]], cur[it.in[2]]), cp.gs2);
  }
  xb[it.out] = o;
}

template <class P, class T>
struct Engine {
  static constexpr int W = MGC_LANES_BYTES / (int)sizeof(T);
  using L = Lane<T, W>;
  using C = mg::cx<L>;
  static constexpr int NC = P::NCOLOR;

  // per-thread work buffers
  std::vector<mg::W4<L>> cur = std::vector<mg::W4<L>>(P::HS_NSLOT);
  std::vector<mg::W4<L>> xb = std::vector<mg::W4<L>>(P::HS_XCAP);
  std::vector<C> J;
  L K[P::NMOM * 4];
  C pr[P::NPROP];

  static mg::Couplings<L> lanes(const mg::Couplings<double>& c) {
    return {L(c.gs), L(c.gs2), L(c.ee), L(c.gz), L(c.gzl), L(c.gzr), L(c.mt)};
  }

  // events [e0, e0 + n), n <= W (missing lanes repeat the last event)
  void block(const double* mom, int64_t nevt, int64_t e0, int n, const int* good, int ng, const mg::PhysParams& pp,
             const mg::Couplings<double>& cd, const mg::Couplings<L>& cl, double* me) {
    using namespace mg;
    double p[P::NPAR][4][W];
    for (int l = 0; l < P::NPAR; ++l)
      for (int mu = 0; mu < 4; ++mu)
        for (int i = 0; i < W; ++i) p[l][mu][i] = mom[(int64_t)(l * 4 + mu) * nevt + e0 + std::min(i, n - 1)];
    // momentum table (FP64 sums of signed external momenta) and propagators
    double Kd[P::NMOM][4][W];
    for (int j = 0; j < P::NMOM; ++j)
      for (int mu = 0; mu < 4; ++mu)
        for (int i = 0; i < W; ++i) {
          double k = 0.0;
          bool first = true;
          for (int l = 0; l < P::NPAR; ++l) {
            if (!(P::mom(j, 1) >> l & 1)) continue;
            const bool neg = P::mom(j, 0) == 1 && (P::mom(j, 2) >> l & 1);
            k = first ? (neg ? -p[l][mu][i] : p[l][mu][i]) : (neg ? k - p[l][mu][i] : k + p[l][mu][i]);
            first = false;
          }
          Kd[j][mu][i] = k;
          K[j * 4 + mu].v[i] = (T)k;
        }
    for (int j = 0; j < P::NPROP; ++j)
      for (int i = 0; i < W; ++i) {
        const double kk[4] = {Kd[P::prop(j, 0)][0][i], Kd[P::prop(j, 0)][1][i], Kd[P::prop(j, 0)][2][i],
                              Kd[P::prop(j, 0)][3][i]};
        double re, im;
        propagator_fp64(kk, P::prop(j, 1), pp, re, im);
        pr[j].re.v[i] = (T)re;
        pr[j].im.v[i] = (T)im;
      }
    // external wavefunctions (level 0) per event in FP64
    const HsItem* items = P::hs_items();
    for (int t = 0; t < P::hs_level(1); ++t) {
      const HsItem& it = items[t];
      W4<L>& o = cur[it.out];
      for (int i = 0; i < W; ++i) {
        const double k[4] = {p[it.a][0][i], p[it.a][1][i], p[it.a][2][i], p[it.a][3][i]};
        const W4<double> w = external<P>(it, k, cd.mt);
        for (int c = 0; c < 4; ++c) {
          o.w[c].re.v[i] = (T)w.w[c].re;
          o.w[c].im.v[i] = (T)w.w[c].im;
        }
      }
    }
    // current variants, level by level
    for (int l = 1; l < P::HS_NLEVEL; ++l)
      for (int t = P::hs_level(l); t < P::hs_level(l + 1); ++t) item<P, L>(items[t], cur.data(), K, pr, cl);
    // amputated currents chunk by chunk; contractions of every good helicity
    J.assign((size_t)ng * NC, C(L(0.0), L(0.0)));
    const uint8_t* vt = P::hs_variants();
    for (int c = 0; c < P::HS_NXCHUNK; ++c) {
      for (int t = P::hs_xitem(c); t < P::hs_xitem(c + 1); ++t) xitem<P, L>(items[t], cur.data(), xb.data(), K, cl);
      for (int h = 0; h < ng; ++h)
        P::template hs_contract<L>(c, SlotArray<L>{cur.data()}, SlotArray<L>{xb.data()}, vt + good[h], &J[(size_t)h * NC]);
    }
    // colour sum per helicity (lane precision), helicity sum per event in FP64
    double sum[W] = {};
    for (int h = 0; h < ng; ++h) {
      const C* Jh = &J[(size_t)h * NC];
      L s(0.0);
      for (int a = 0; a < NC; ++a) {
        L ur(0.0), ui(0.0);
        for (int b = 0; b < NC; ++b) {
          const int cn = P::cnum(a, b);
          if (cn == 0) continue;
          const L cv((double)cn);
          ur = fmac(cv, Jh[b].re, ur);
          ui = fmac(cv, Jh[b].im, ui);
        }
        s = fmac(Jh[a].re, ur, fmac(Jh[a].im, ui, s));
      }
      for (int i = 0; i < W; ++i) sum[i] += (double)s.v[i] / (double)P::CDEN;
    }
    for (int i = 0; i < n; ++i) me[e0 + i] = sum[i] * P::NORM;
  }
};

template <class P, class T>
void run(int64_t nevt, const double* mom, const int32_t* mask, const mg_params& prm, double* me, int nthreads) {
  using E = Engine<P, T>;
  int good[64];
  int ng = 0;
  for (int h = 0; h < P::NHEL; ++h)
    if (mask[h] != 0) good[ng++] = h;
  const mg::PhysParams pp{prm.mz, prm.wz, prm.mt, prm.wt};
  mg::Couplings<double> cd;
  const double e = std::sqrt(4.0 * M_PI / prm.alpha_inv), gs = std::sqrt(4.0 * M_PI * prm.alpha_s);
  cd.gs = gs;
  cd.gs2 = gs * gs;
  cd.ee = e;
  cd.gz = e / std::sqrt(prm.sw2 * (1.0 - prm.sw2));
  cd.gzl = -0.5 + prm.sw2;
  cd.gzr = prm.sw2;
  cd.mt = prm.mt;
  if (ng == 0) {
    std::fill(me, me + nevt, 0.0);
    return;
  }
  const int64_t nblk = (nevt + E::W - 1) / E::W;
  auto work = [&](int64_t b0, int64_t b1) {
    E eng;
    const auto cl = E::lanes(cd);
    for (int64_t b = b0; b < b1; ++b) {
      const int64_t e0 = b * E::W;
      const int n = (int)std::min<int64_t>(E::W, nevt - e0);
      eng.block(mom, nevt, e0, n, good, ng, pp, cd, cl, me);
    }
  };
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, nblk));
  if (nt == 1) {
    work(0, nblk);
    return;
  }
  std::vector<std::thread> th;
  const int64_t per = (nblk + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int64_t b0 = t * per, b1 = std::min(nblk, b0 + per);
    if (b0 < b1) th.emplace_back(work, b0, b1);
  }
  for (auto& x : th) x.join();
}

template <class T>
int dispatch(int proc, int64_t nevt, const double* mom, const int32_t* mask, const mg_params& prm, double* me,
             int nthreads) {
  switch (proc) {
    case 1: run<mg::Proc1, T>(nevt, mom, mask, prm, me, nthreads); return MG_OK;
    case 2: run<mg::Proc2, T>(nevt, mom, mask, prm, me, nthreads); return MG_OK;
    case 3: run<mg::Proc3, T>(nevt, mom, mask, prm, me, nthreads); return MG_OK;
    case 4: run<mg::Proc4, T>(nevt, mom, mask, prm, me, nthreads); return MG_OK;
  }
  return MG_ERR_PROC;
}

}  // namespace mgcpu

extern "C" {

int mgc_lanes(int precision) { return MGC_LANES_BYTES / (precision == 0 ? 8 : 4); }

int mgc_sigmakin(int proc, int64_t nevt, const double* mom, const int32_t* mask, int precision,
                 const mg_params* params, double* me, int nthreads) {
  if (proc < 1 || proc > 4) return MG_ERR_PROC;
  if (nevt < 0 || (precision != 0 && precision != 1) || nthreads < 1) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!mom || !mask || !me || !params) return MG_ERR_ARG;
  const mg_params prm = *params;
  return precision == 0 ? mgcpu::dispatch<double>(proc, nevt, mom, mask, prm, me, nthreads)
                        : mgcpu::dispatch<float>(proc, nevt, mom, mask, prm, me, nthreads);
}

}  // extern "C"
