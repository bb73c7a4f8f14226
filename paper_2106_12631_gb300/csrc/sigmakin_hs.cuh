// SIGMAKIN with helicity-shared currents (the default kernel of both modes).
//
// Same result as the straight-line kernel (sigmakin.cuh) — the same Feynman
// diagrams, colour flows and colour matrix (Sec. 2) — organised for GB300:
//   * an off-shell current over legs S depends only on the helicities of S,
//     so each current is computed once per event for each of its 2^|S|
//     helicity variants (not once per event helicity), into shared memory;
//   * every diagram's amplitude is formed at a vertex chosen by the generator,
//     with one operand Y left out: A = sum_i X_i Y_i, where the amputated
//     current X of the other operands is again shared across helicities;
//   * currents and amputated currents are item tables walked by short loops
//     (lanes take one item for each of the CTA's events); the contractions of
//     a chunk's amplitudes are generated straight-line code.
// CTA of NT threads = EV events x ngood helicities.  Phases:
//   1. per-event momenta, momentum sums and FP64 propagator factors (as SIGMAKIN);
//   2. current variants, level by level (a level only reads earlier levels);
//   3. per chunk of amputated currents: their variants (all threads), then one
//      thread per (event, helicity) contracts the chunk's amplitudes and adds
//      each into its colour flows J (registers);
//   4. colour sum (CUDA cores, or tcgen05 as in sigmakin.cuh) and the
//      fixed-order FP64 helicity sum.
#pragma once
#include <type_traits>

#include "rambo.cuh"
#include "rng.cuh"
#include "sigmakin.cuh"

namespace mg {

#ifndef MG_HS_NT
#define MG_HS_NT 256
#endif
#ifndef MG_HS_CTAS
#define MG_HS_CTAS 2  // resident CTAs per SM the shared-memory budget is split for (24+ colour flows)
#endif
#ifndef MG_HS_EVENT_SYNC
#define MG_HS_EVENT_SYNC 0  // 1: per-event barrier groups (HsGroup) instead of CTA barriers
#endif
#ifndef MG_HS_CTAS_SMALL
#define MG_HS_CTAS_SMALL 3  // the same below 24 colour flows (smaller variant sets per event)
#endif

// Many-colour processes in FP32: several 256-thread CTAs per SM (two of
// 4 events x 64 helicities for gg -> t t~ g g, three of 8 x 32 for
// gg -> t t~ g), so that one CTA's short barrier-bound phases overlap the
// others' contractions (measured).  FP64 needs more registers per thread:
// one 256-thread CTA per SM.
template <class P, class R>
struct HsCfg {
  static constexpr int NT = P::NCOLOR >= 6 ? (sizeof(R) == 4 ? MG_HS_NT : 256) : 128;
  static constexpr int EVMIN = (NT / P::NHEL) > 0 ? (NT / P::NHEL) : 1;
  static constexpr int EVWANT = (4 * EVMIN) < 32 ? 4 * EVMIN : 32;
  // shared memory for the current variants and one chunk of amputated currents
  static constexpr int CTAS =
      P::NCOLOR >= 6 && sizeof(R) == 4 ? (P::NCOLOR >= 24 ? MG_HS_CTAS : MG_HS_CTAS_SMALL) : 1;
  static constexpr size_t CUR_BUDGET = 192 * 1024 / CTAS;
  static constexpr size_t EV_BYTES = (size_t)(P::HS_NSLOT + P::HS_XBUFS * P::HS_XCAP) * sizeof(W4<R>);
  static constexpr int FIT = (int)(CUR_BUDGET / EV_BYTES);
  static constexpr int EVCAP = FIT < EVWANT ? (FIT > EVMIN ? FIT : EVMIN) : EVWANT;
  static constexpr int KP = ((P::NCOLOR + 15) / 16) * 16;
  static constexpr int NP = KP;
  static constexpr int MBLK = NT / 128;
};

template <class P, class R, int CS>
struct HsLayout {
  using H = HsCfg<P, R>;
  static constexpr int NT = H::NT, EVCAP = H::EVCAP, KP = H::KP, NP = H::NP, MBLK = H::MBLK;
  static constexpr bool TC = CS == CS_TC;
  static constexpr size_t o_proptab = 0;  // {momentum entry, line kind} per propagator
  static constexpr size_t o_md = align_up(o_proptab + 8 * P::NPROP, 16);  // momentum-entry descriptors (int4)
  static constexpr size_t o_good = align_up(o_md + 16 * P::NMOM, 16);
  static constexpr size_t o_misc = align_up(o_good + 4 * P::NHEL, 16);
  // mixed mode: {m^2 hi, m^2 lo, m w, 0} of the top and of the Z
  static constexpr size_t o_mconst = align_up(o_misc + 32, 16);
  static constexpr size_t o_p = align_up(o_mconst + 32, 16);
  // the next group's momenta (FP64), copied asynchronously while this group runs
  static constexpr size_t o_ps = align_up(o_p + 8 * EVCAP * P::NPAR * 4, 16);
  static constexpr size_t o_K = align_up(o_ps + 8 * EVCAP * P::NPAR * 4, 16);
  // momentum-table entries (R) from one event to the next: an odd number of
  // 16-byte words, so that one entry of the CTA's events falls in different
  // bank groups (the lanes of a warp read it for several events at once)
  static constexpr int KEV =
      4 * P::NMOM + ((4 * P::NMOM * (int)sizeof(R) / 16) % 2 == 0 ? 16 / (int)sizeof(R) : 0);
  static constexpr size_t o_pr = align_up(o_K + sizeof(R) * EVCAP * KEV, 16);
  static constexpr size_t o_m2 = align_up(o_pr + 2 * sizeof(R) * EVCAP * P::NPROP, 16);
  // variant of a leg set for a helicity: vt[S * NHEL + ihel]
  static constexpr size_t o_vt = align_up(o_m2 + 8 * NT, 16);
  static constexpr size_t o_U = align_up(o_vt + (size_t(1) << P::NPAR) * P::NHEL, 1024);
  // union: current variants + amputated chunk (phases 2-3), then the tensor-core
  // A tiles and, after them, the colour matrix as the B operand (phase 4).
  // Per-event strides in 16-byte words, padded so that one slot of the CTA's
  // events falls in different bank groups: the lanes of a warp take an item
  // for several events at once (the plane stride, a multiple of 8 words for
  // the processes' slot counts, would otherwise map them to one group).
  static constexpr int EVPAD = EVCAP >= 8 ? 1 : 8 / EVCAP;
  static constexpr int CUR_EV = P::HS_NSLOT * Slots<R, 1>::NPL + EVPAD;
  static constexpr int X_EV = P::HS_XCAP * Slots<R, 1>::NPL + EVPAD;
  static constexpr size_t o_cur = o_U;
  static constexpr size_t o_x = o_U + 16 * size_t(EVCAP) * CUR_EV;
  static constexpr size_t o_A = o_U;
  static constexpr size_t tileA = 128 * KP * 2;
  static constexpr size_t u_bytes = 16 * size_t(EVCAP) * (CUR_EV + P::HS_XBUFS * X_EV);
  static constexpr size_t a_bytes = TC ? 3 * MBLK * tileA : 0;  // one component's three splits
  static constexpr size_t o_B = o_U + a_bytes;  // copied in for every group's colour sum
  static constexpr size_t b_bytes = TC ? size_t(NP) * KP * 2 : 0;
  static constexpr size_t bytes = o_U + (u_bytes > a_bytes + b_bytes ? u_bytes : a_bytes + b_bytes);
  static_assert(o_B % 1024 == 0, "B operand on a 1024-byte boundary");
  static constexpr uint32_t TMEM_COLS = tc::tmem_cols(MBLK * 2 * NP);
  static_assert(!TC || NT % 128 == 0, "CTA rows must fill 128-row MMA blocks");
  static_assert(TMEM_COLS <= 512, "TMEM holds 512 columns");
  static_assert(bytes <= 232448, "shared memory per CTA above the 227 KB limit");
};

// Tensor-core colour sum of the CTA's NT rows with J in registers (layout and
// three-term BF16 split as in colour_tc.cuh).  Two passes, real then imaginary
// part, so that one component's A tiles fit in the dead current-variant
// storage: Y_c = A_c B lands in TMEM columns [c NP, (c+1) NP).
template <class P, class L>
__device__ __forceinline__ float colour_sum_tc_regs(unsigned char* smem, const cx<float>* J, uint32_t tmem,
                                                    uint32_t mbar) {
  constexpr int NC = P::NCOLOR, KP = L::KP;
  const int tid = threadIdx.x;
  const int b = tid >> 7, r = tid & 127;
  bool ok = true;
  {  // the colour matrix (BF16 B operand) into the union, free from here on
    const uint4* src = reinterpret_cast<const uint4*>(P::colour_bf16_image());
    uint4* dst = reinterpret_cast<uint4*>(smem + L::o_B);
    for (int i = tid; i < (int)(L::b_bytes / 16); i += L::NT) dst[i] = src[i];
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c == 1) {
      // pass 0's MMAs have read its tiles once every thread saw the barrier
      // complete; a timed-out wait ends both passes for the whole CTA
      if (__syncthreads_or(!ok)) {
        tc::mbar_wait(mbar, 0);
        return __int_as_float(0x7fc00000);
      }
    }
#pragma unroll
    for (int k0 = 0; k0 < KP; k0 += 8) {
      uint32_t w[3][4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        uint16_t hb[3][2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k = k0 + q + u;
          const float x = k < NC ? (c == 0 ? J[k].re : J[k].im) : 0.0f;
          const uint16_t h = tc::bf16_bits(x);
          const float r1 = x - tc::bf16_value(h);
          const uint16_t m = tc::bf16_bits(r1);
          const uint16_t l = tc::bf16_bits(r1 - tc::bf16_value(m));
          hb[0][u] = h; hb[1][u] = m; hb[2][u] = l;
        }
#pragma unroll
        for (int sp = 0; sp < 3; ++sp) w[sp][q >> 1] = (uint32_t)hb[sp][0] | ((uint32_t)hb[sp][1] << 16);
      }
#pragma unroll
      for (int sp = 0; sp < 3; ++sp) {
        unsigned char* tile = smem + L::o_A + (sp * L::MBLK + b) * L::tileA;
        *reinterpret_cast<uint4*>(tile + tc::kmajor_offset<KP>(r, k0)) =
            make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
      }
    }
    tc::fence_async_shared();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      constexpr uint32_t idesc = tc::idesc_bf16(128, L::NP);
      constexpr uint32_t LBO = 128, SBO = (KP / 8) * 128;
      const uint32_t bbase = tc::smem_addr(smem + L::o_B);
#pragma unroll
      for (int bb = 0; bb < L::MBLK; ++bb) {
        const uint32_t d = tmem + (uint32_t)((bb * 2 + c) * L::NP);
#pragma unroll
        for (int sp = 0; sp < 3; ++sp) {
          const uint32_t abase = tc::smem_addr(smem + L::o_A + (sp * L::MBLK + bb) * L::tileA);
#pragma unroll
          for (int j = 0; j < KP / 16; ++j)
            tc::mma_bf16(d, tc::smem_desc(abase + j * 256, LBO, SBO), tc::smem_desc(bbase + j * 256, LBO, SBO),
                         idesc, (sp | j) != 0);
        }
      }
      tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait(mbar, (uint32_t)c);
  }
  tc::fence_after_sync();
  const int warp = tid >> 5;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  float yr[L::NP], yi[L::NP];
#pragma unroll
  for (int c0 = 0; c0 < L::NP; c0 += 16) {
    tc::tmem_ld16(tmem + lane_base + (uint32_t)((b * 2 + 0) * L::NP + c0), yr + c0);
    tc::tmem_ld16(tmem + lane_base + (uint32_t)((b * 2 + 1) * L::NP + c0), yi + c0);
  }
  tc::tmem_wait_ld();
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < NC; ++k) s += J[k].re * yr[k] + J[k].im * yi[k];
  s *= 1.0f / (float)P::CDEN;
  if (!ok) {
    tc::mbar_wait(mbar, 1);  // second bounded wait for the MMAs still in flight
    s = __int_as_float(0x7fc00000);
  }
  return s;
}

// |M_h|^2 = J^dagger C J / CDEN on CUDA cores with C real symmetric:
//   sum_i J_i^* (C_ii J_i + 2 sum_{j>i} C_ij J_j)  (real part; the imaginary parts cancel)
// — each off-diagonal entry once, half the multiply-adds of the row-wise form.
template <class P>
__host__ __device__ constexpr bool colour_matrix_symmetric() {
  for (int i = 0; i < P::NCOLOR; ++i)
    for (int j = 0; j < i; ++j)
      if (P::cnum(i, j) != P::cnum(j, i)) return false;
  return true;
}
// f(std::integral_constant<int, i>) for i = B .. E - 1: indices that are
// compile-time constants by construction (the colour matrix entries below are
// then immediates, whatever the unroller decides inside a large loop body)
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

template <class P, class R>
__device__ __forceinline__ R colour_sum_sym(const cx<R>* J) {
  static_assert(colour_matrix_symmetric<P>(), "colour matrix must be symmetric");
  constexpr int NC = P::NCOLOR;
  if constexpr (sizeof(R) == 4) {
    // FP32: the real and imaginary parts side by side in the paired FP32
    // instructions (one FFMA2 per matrix entry instead of two FFMAs)
    float2 tot = make_float2(0.0f, 0.0f);
    static_for<0, NC>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr float cii = (float)P::cnum(i, i);
      float2 u = __fmul2_rn(make_float2(cii, cii), make_float2(J[i].re, J[i].im));
      static_for<i + 1, NC>([&](auto Jc) {
        constexpr int j = decltype(Jc)::value;
        if constexpr (P::cnum(i, j) != 0) {
          constexpr float c = (float)(2 * P::cnum(i, j));
          u = __ffma2_rn(make_float2(c, c), make_float2(J[j].re, J[j].im), u);
        }
      });
      tot = __ffma2_rn(make_float2(J[i].re, J[i].im), u, tot);
    });
    return (tot.x + tot.y) / R(P::CDEN);
  }
  R sum = R(0);
  static_for<0, NC>([&](auto I) {
    constexpr int i = decltype(I)::value;
    R ur = R(P::cnum(i, i)) * J[i].re, ui = R(P::cnum(i, i)) * J[i].im;
    static_for<i + 1, NC>([&](auto Jc) {
      constexpr int j = decltype(Jc)::value;
      if constexpr (P::cnum(i, j) != 0) {
        ur += R(2 * P::cnum(i, j)) * J[j].re;
        ui += R(2 * P::cnum(i, j)) * J[j].im;
      }
    });
    sum = fmac(J[i].re, ur, fmac(J[i].im, ui, sum));
  });
  return sum / R(P::CDEN);
}

// Propagator factor of one line from its FP64 momentum: the invariant
// k^2 - m^2 is formed in FP64 (it cancels near the pole and for collinear
// pairs); the reciprocal 1/(k^2 - m^2 + i m w) times i (fermion) or -i (vector)
// is taken in the working precision.
template <class R>
__device__ __forceinline__ cx<R> propagator_hs(const double* k, int kind, const PhysParams& pp) {
  const double k2 = k[0] * k[0] - k[1] * k[1] - k[2] * k[2] - k[3] * k[3];
  double dr = k2, di = 0.0;
  if (kind == 1) { dr = k2 - pp.mt * pp.mt; di = pp.mt * pp.wt; }
  else if (kind == 3) { dr = k2 - pp.mz * pp.mz; di = pp.mz * pp.wz; }
  const R r = R(dr), i = R(di);
  const R inv = R(1) / (r * r + i * i);
  const R ar = r * inv, ai = -i * inv;
  return kind == 1 ? cx<R>(-ai, ar) : cx<R>(ai, -ar);
}

// ---- double-float arithmetic for the mixed mode ---------------------------------
// A value as an unevaluated sum hi + lo of two FP32 numbers.  Sums use Knuth's
// error-free TwoSum (the rounding error of a + b is exactly representable and
// recovered with six additions) accumulated as in the cascaded summation of
// Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005); squares use the
// FMA-based exact product.  The result is as accurate as a sum evaluated in
// twice the FP32 precision and then rounded — ample for momentum sums rounded
// to FP32 and for k^2 - m^2 near a pole — while GB300 runs FP32 at 64 times its
// FP64 rate.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl dfl_split(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
// sum of signed terms t_k = hi_k + lo_k, k = 0..n-1
struct DflSum {
  float s, err;
  __device__ __forceinline__ void first(float hi, float lo) { s = hi; err = lo; }
  __device__ __forceinline__ void add(float hi, float lo) {
    const dfl t = two_sum(s, hi);
    s = t.hi;
    err += t.lo + lo;
  }
  __device__ __forceinline__ float value() const { return s + err; }
};

// Propagator factor from a double-float momentum: k^2 - m^2 summed error-free
// from the exact squares of the components, then the reciprocal in FP32.
// m2 = m^2 as double-float, mw = m w.
__device__ __forceinline__ cx<float> propagator_dfl(const float2* k, int kind, dfl m2, float mw) {
  DflSum d;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const float h = k[mu].x, l = k[mu].y;
    const float p = h * h;
    float e = fmaf(h, h, -p);
    e = fmaf(2.0f * h, l, e);
    if (mu == 0) d.first(p, e);
    else d.add(-p, -e);
  }
  float di = 0.0f;
  if (kind == 1 || kind == 3) {
    d.add(-m2.hi, -m2.lo);
    di = mw;
  }
  const float r = d.value();
  const float inv = 1.0f / (r * r + di * di);
  const float ar = r * inv, ai = -di * inv;
  return kind == 1 ? cx<float>(-ai, ar) : cx<float>(ai, -ar);
}

// Phase 1 of the forward kernels, in three parts:
//   hs_setup_words   per-CTA constants: {momentum entry, line kind} per
//                    propagator, a descriptor per momentum-table entry, and in
//                    the mixed mode {m^2 hi, m^2 lo, m w, 0} of the top and Z;
//   hs_load_momenta  the CTA's momenta into shared memory: FP64, or in the
//                    mixed mode each component split into a double-float pair;
//   hs_tables        (after a barrier) one thread per (event, momentum-table
//                    entry) sums the entry's signed external momenta — in FP64
//                    (FP64 mode) or double-float (mixed mode), every leg in leg
//                    order with coefficient +1, -1 or 0 (adding an exact zero
//                    changes neither an FP64 sum nor a double-float pair), rounds
//                    it to R for the currents and forms the propagator factor
//                    of every line with that momentum from the unrounded sum;
//                    one thread per (event, external leg variant) builds the
//                    external wavefunction (level 0 of the current program).

// Descriptor of momentum-table entry j: {legs added, legs subtracted, first
// propagator on that momentum, second} (-1: none).
template <class P>
__device__ __forceinline__ int4 hs_mom_desc(int j) {
  int4 v = make_int4(0, 0, -1, -1);
#pragma unroll
  for (int jj = 0; jj < P::NMOM; ++jj) {
    if (j != jj) continue;
    const int legs = P::mom(jj, 1), neg = P::mom(jj, 0) == 1 ? (P::mom(jj, 2) & legs) : 0;
    v = make_int4(legs & ~neg, neg, P::mom_prop(jj, 0), P::mom_prop(jj, 1));
  }
  return v;
}

template <class P, class R, class L>
__device__ __forceinline__ void hs_setup_words(unsigned char* smem, const PhysParams& pp) {
  static_assert(L::NT >= P::NPROP && L::NT >= P::NMOM, "one thread per propagator and per momentum entry");
  const int tid = threadIdx.x;
  if (tid < P::NPROP) {
    int2 v = make_int2(0, 0);
#pragma unroll
    for (int j = 0; j < P::NPROP; ++j)
      if (tid == j) v = make_int2(P::prop(j, 0), P::prop(j, 1));
    reinterpret_cast<int2*>(smem + L::o_proptab)[tid] = v;
  }
  if (tid < P::NMOM) reinterpret_cast<int4*>(smem + L::o_md)[tid] = hs_mom_desc<P>(tid);
  if constexpr (sizeof(R) == 4) {
    if (tid < 2) {
      const double m = tid == 0 ? pp.mt : pp.mz, w = tid == 0 ? pp.wt : pp.wz;
      const dfl m2 = dfl_split(m * m);
      reinterpret_cast<float4*>(smem + L::o_mconst)[tid] = make_float4(m2.hi, m2.lo, (float)(m * w), 0.0f);
    }
  }
}

// p[e][leg][mu]: double, or float2 (hi, lo) in the mixed mode (same 8 bytes)
template <class P, class R, class L>
__device__ __forceinline__ void hs_load_momenta(unsigned char* smem, const double* __restrict__ mom, int64_t nevt,
                                                int64_t e0, int nev) {
  for (int t = threadIdx.x; t < nev * P::NPAR * 4; t += L::NT) {
    const int e = t % nev, c = t / nev;
    const double x = mom[(int64_t)c * nevt + e0 + e];
    if constexpr (sizeof(R) == 4) {
      const dfl q = dfl_split(x);
      reinterpret_cast<float2*>(smem + L::o_p)[e * P::NPAR * 4 + c] = make_float2(q.hi, q.lo);
    } else {
      reinterpret_cast<double*>(smem + L::o_p)[e * P::NPAR * 4 + c] = x;
    }
  }
}

// A later group's momenta, copied asynchronously (cp.async, 8 bytes per
// component) into the staging buffer in the layout of p; the copies of each
// thread complete at its cp_async_wait_all, and hs_convert_momenta (after a
// barrier) turns them into p.
template <class P, class L>
__device__ __forceinline__ void hs_prefetch_momenta(unsigned char* smem, const double* __restrict__ mom, int64_t nevt,
                                                    int64_t e0, int nev) {
  const uint32_t st = tc::smem_addr(smem + L::o_ps);
  for (int t = threadIdx.x; t < nev * P::NPAR * 4; t += L::NT) {
    const int e = t % nev, c = t / nev;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(st + 8u * (uint32_t)(e * P::NPAR * 4 + c)),
                 "l"(mom + (int64_t)c * nevt + e0 + e)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class P, class R, class L>
__device__ __forceinline__ void hs_convert_momenta(unsigned char* smem, int nev) {
  const double* st = reinterpret_cast<const double*>(smem + L::o_ps);
  for (int t = threadIdx.x; t < nev * P::NPAR * 4; t += L::NT) {
    const double x = st[t];
    if constexpr (sizeof(R) == 4) {
      const dfl q = dfl_split(x);
      reinterpret_cast<float2*>(smem + L::o_p)[t] = make_float2(q.hi, q.lo);
    } else {
      reinterpret_cast<double*>(smem + L::o_p)[t] = x;
    }
  }
}

// Barrier domain of the phases after the CTA's first barrier: the threads of
// one event, or of the events that share one warp, synchronise only among
// themselves, so the events of a CTA move through their phases independently.
// With ng good helicities (thread = (event, good helicity)): ng = 64 -> one
// event per two warps on a named barrier; ng = 32 -> one event per warp; ng a
// divisor of 32 -> the 32 / ng events of one warp; otherwise, and for the
// tensor-core colour sum (one MMA spans several events), the whole CTA.
struct HsGroup {
  int kind;      // 0 CTA barrier, 1 warp, 2 named barrier
  int tpg;       // threads per group
  int j;         // thread index within the group
  int ev0, nev;  // the group's events (CTA-local)
  int id;        // named barrier (kind 2)
  __device__ __forceinline__ void sync() const {
    if (kind == 0) __syncthreads();
    else if (kind == 1) __syncwarp();
    else named_sync();
  }
  // barrier ids as immediates, so only the ids in use are reserved
  __device__ __forceinline__ void named_sync() const {
    switch (id) {
      case 1: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
      case 2: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
      case 3: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
      case 4: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
      case 5: asm volatile("bar.sync 5, 64;" ::: "memory"); break;
      case 6: asm volatile("bar.sync 6, 64;" ::: "memory"); break;
      case 7: asm volatile("bar.sync 7, 64;" ::: "memory"); break;
      default: asm volatile("bar.sync 8, 64;" ::: "memory"); break;
    }
  }
};

template <int NT>
__device__ __forceinline__ HsGroup hs_group(bool cta_only, int ng, int ev, int nev) {
  static_assert(NT % 64 == 0 && NT / 64 <= 8, "named barriers 1..8 for the two-warp groups");
  HsGroup g;
  int epg;
  if (cta_only || ng < 1 || !(ng == 64 || 32 % ng == 0)) {
    g.kind = 0;
    g.tpg = NT;
    epg = ev;
  } else if (ng == 64) {
    g.kind = 2;
    g.tpg = 64;
    epg = 1;
  } else {
    g.kind = 1;
    g.tpg = 32;
    epg = 32 / ng;
  }
  const int grp = (int)threadIdx.x / g.tpg;
  g.j = (int)threadIdx.x - grp * g.tpg;
  g.ev0 = grp * epg;
  g.nev = max(0, min(epg, nev - g.ev0));
  g.id = 1 + grp;
  return g;
}

// CUR_EV: 16-byte words from one event's current variants to the next's;
// KEV: momentum-table entries (R) from one event's table to the next's
template <class P, class R, class L, int CUR_EV = P::HS_NSLOT * Slots<R, 1>::NPL, int KEV = 4 * P::NMOM>
__device__ __forceinline__ void hs_tables(unsigned char* smem, const PhysParams& pp, const HsGroup& grp, uint4* curs,
                                          const Couplings<R>& cp) {
  constexpr int NM = P::NMOM, NPAR = P::NPAR;
  constexpr int NEXT = P::hs_level(1);  // external variants
  constexpr bool DF = sizeof(R) == 4;
  const int4* md = reinterpret_cast<const int4*>(smem + L::o_md);
  const int2* prop_tab = reinterpret_cast<const int2*>(smem + L::o_proptab);
  R* K = reinterpret_cast<R*>(smem + L::o_K);                // [EV][NMOM][4]
  cx<R>* pr = reinterpret_cast<cx<R>*>(smem + L::o_pr);      // [EV][NPROP]
  const int nev = grp.nev;
  for (int t = grp.j; t < nev * (NM + NEXT); t += grp.tpg) {
    if (t < nev * NM) {
      const int el = t / NM, j = t - el * NM, e = grp.ev0 + el;
      const int4 d = md[j];
      if constexpr (DF) {
        const float2* q = reinterpret_cast<const float2*>(smem + L::o_p) + e * NPAR * 4;
        float2 kf[4];
        float kv[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          DflSum k;
          k.first(0.0f, 0.0f);
#pragma unroll
          for (int l = 0; l < NPAR; ++l) {
            const float2 v = q[l * 4 + mu];
            const float c = (d.x >> l & 1) ? 1.0f : ((d.y >> l & 1) ? -1.0f : 0.0f);
            k.add(c * v.x, c * v.y);
          }
          kf[mu] = make_float2(k.s, k.err);
          kv[mu] = k.value();
        }
        *reinterpret_cast<float4*>(K + e * KEV + 4 * j) = make_float4(kv[0], kv[1], kv[2], kv[3]);
        const float4* mc = reinterpret_cast<const float4*>(smem + L::o_mconst);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int pj = u == 0 ? d.z : d.w;
          if (pj < 0) continue;
          const int kind = prop_tab[pj].y;
          const float4 c = mc[kind == 3 ? 1 : 0];  // {m^2 hi, m^2 lo, m w, 0} of the top / the Z
          pr[e * P::NPROP + pj] = propagator_dfl(kf, kind, dfl{c.x, c.y}, c.z);
        }
      } else {
        const double* q = reinterpret_cast<const double*>(smem + L::o_p) + e * NPAR * 4;
        double k[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          double s = 0.0;
#pragma unroll
          for (int l = 0; l < NPAR; ++l) {
            const double c = (d.x >> l & 1) ? 1.0 : ((d.y >> l & 1) ? -1.0 : 0.0);
            s += c * q[l * 4 + mu];
          }
          k[mu] = s;
          K[e * KEV + j * 4 + mu] = R(s);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int pj = u == 0 ? d.z : d.w;
          if (pj < 0) continue;
          pr[e * P::NPROP + pj] = propagator_hs<R>(k, prop_tab[pj].y, pp);
        }
      }
    } else {
      const int t2 = t - nev * NM, el = t2 / NEXT, e = grp.ev0 + el;
      const HsItem it = P::hs_items()[t2 - el * NEXT];
      R k[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        if constexpr (DF) k[mu] = reinterpret_cast<const float2*>(smem + L::o_p)[(e * NPAR + it.a) * 4 + mu].x;
        else k[mu] = reinterpret_cast<const double*>(smem + L::o_p)[(e * NPAR + it.a) * 4 + mu];
      }
      W4<R> o;
      if (it.type == 0) o = ixxxxx<R>(k, it.flag ? cp.mt : R(0), it.b, it.c);
      else if (it.type == 1) o = oxxxxx<R>(k, it.flag ? cp.mt : R(0), it.b, it.c);
      else o = vxxxxx<R>(k, it.b, it.c);
      Slots<R, P::HS_NSLOT>{curs + e * CUR_EV}.set(it.out, o);
    }
  }
  grp.sync();
}

// Item of work index t when the lanes take items item-major: consecutive
// lanes take one item for each of the group's nev events, so that a warp holds
// 32 / nev items (of one vertex type wherever the generator's per-event type
// segments are multiples of that) and reads each descriptor once for all
// its events.
template <class L>
__device__ __forceinline__ int hs_item_of(int t, int nev) {
  return nev == L::EVCAP ? t / L::EVCAP : t / nev;
}

// one current variant
template <class P, class R>
__device__ __forceinline__ void hs_item(const HsItem& it, const Slots<R, P::HS_NSLOT>& cur, const R* K,
                                        const cx<R>* pr, const Couplings<R>& cp) {
  W4<R> o;
  switch (it.type) {
    case 0: o = ixxxxx<R>(K + 4 * it.k0, it.flag ? cp.mt : R(0), it.b, it.c); break;
    case 1: o = oxxxxx<R>(K + 4 * it.k0, it.flag ? cp.mt : R(0), it.b, it.c); break;
    case 2: o = vxxxxx<R>(K + 4 * it.k0, it.b, it.c); break;
    case 3: o = FFV1_2<R>(cur[it.in[0]], cur[it.in[1]], cp.gs, K + 4 * it.k0, cp.mt, pr[it.prop]); break;
    case 4: o = FFV1_1<R>(cur[it.in[0]], cur[it.in[1]], cp.gs, K + 4 * it.k0, cp.mt, pr[it.prop]); break;
    case 5: o = FFV1P0_3<R>(cur[it.in[0]], cur[it.in[1]], it.a ? cp.ee : cp.gs, pr[it.prop]); break;
    case 6: o = FFV2_4_3<R>(cur[it.in[0]], cur[it.in[1]], cp.gz, cp.gzl, cp.gzr, pr[it.prop]); break;
    case 7: o = VVV1P0_1<R>(cur[it.in[0]], cur[it.in[1]], K + 4 * it.k0, K + 4 * it.k1, cp.gs, pr[it.prop]); break;
    default: {  // four-gluon term X_0 (X_1 . W) - X_1 (X_0 . W), in = {X_0, X_1, W}
      const W4<R> x0 = cur[it.in[0]], x1 = cur[it.in[1]], w = cur[it.in[2]];
      o = vvvv_comb(x0, vdot(x1, w), x1, vdot(x0, w), mul_mi(cp.gs2 * pr[it.prop]));
    }
  }
  cur.set(it.out, o);
}

// one amputated-current variant (reads the currents, writes the chunk buffer)
template <class P, class R>
__device__ __forceinline__ void hs_xitem(const HsItem& it, const Slots<R, P::HS_NSLOT>& cur,
                                         const Slots<R, P::HS_XCAP>& xb, const R* K, const Couplings<R>& cp) {
  W4<R> o;
  switch (it.type) {
    case 9: o = FFV1_2A<R>(cur[it.in[0]], cur[it.in[1]], cp.gs); break;
    case 10: o = FFV1_1A<R>(cur[it.in[0]], cur[it.in[1]], cp.gs); break;
    case 11: o = FFV1P0_3A<R>(cur[it.in[0]], cur[it.in[1]], it.a ? cp.ee : cp.gs); break;
    case 12: o = FFV2_4_3A<R>(cur[it.in[0]], cur[it.in[1]], cp.gz, cp.gzl, cp.gzr); break;
    case 13: o = VVV1P0_1A<R>(cur[it.in[0]], cur[it.in[1]], K + 4 * it.k0, K + 4 * it.k1, cp.gs); break;
    default: {  // four-gluon term, as in hs_item
      const W4<R> x0 = cur[it.in[0]], x1 = cur[it.in[1]], w = cur[it.in[2]];
      o = vvvv_comb_a(x0, vdot(x1, w), x1, vdot(x0, w), cp.gs2);
    }
  }
  xb.set(it.out, o);
}

// Inverse-CDF sampling by one warp: the first k < n, in order, whose running
// sum of the weights get(k) exceeds u * (their total), the last one if
// rounding leaves none, -1 if the total is not positive (FP64; n <= 32 RND,
// lanes take consecutive k, running sums by warp scans 32 weights at a time,
// the total is the last running sum).
template <int RND, class F>
__device__ __forceinline__ int warp_inverse_cdf(int n, double u, int lane, F get) {
  double run[RND];
  double carry = 0.0;
#pragma unroll
  for (int r = 0; r < RND; ++r) {
    run[r] = 0.0;
    if (32 * r < n) {
      double x = 32 * r + lane < n ? get(32 * r + lane) : 0.0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      run[r] = carry + x;
      carry = __shfl_sync(0xffffffffu, run[r], 31);
    }
  }
  if (!(carry > 0.0)) return -1;
  const double target = u * carry;
#pragma unroll
  for (int r = 0; r < RND; ++r) {
    const unsigned hit = __ballot_sync(0xffffffffu, 32 * r + lane < n && run[r] > target);
    if (hit) return 32 * r + __ffs(hit) - 1;
  }
  return n - 1;
}

// Per event: a good helicity with probability |M_h|^2 / sum (weights sm2 of
// the event's threads, helicity order) and a colour flow s with probability
// w_s / sum, w_s = sum over the good helicities of |J_s|^2; one warp per event.
// The |J_s|^2 of every thread are staged in the dead union region, thread-major
// with an odd row stride (lane s of the event's warp sums row entries s over
// the event's helicities, in helicity order, in the working precision; the
// running sums that decide are FP64).
template <class P, class R>
struct HsChoice {
  static constexpr int NCP = P::NCOLOR | 1;
};

template <class P, class R, class L>
__device__ __forceinline__ void hs_choices(const unsigned char* smem, const SigArgs& a, int64_t e0, int nev, int ng,
                                           const int* good, const double* sm2) {
  constexpr int NT = L::NT, NC = P::NCOLOR, NCP = HsChoice<P, R>::NCP;
  static_assert(NC <= 32, "one lane per colour flow");
  static_assert(sizeof(R) * NCP * NT <= L::u_bytes, "colour weights overflow their scratch");
  const int tid = threadIdx.x, lane = tid & 31;
  const R* wj = reinterpret_cast<const R*>(smem + L::o_U);
  for (int e = tid >> 5; e < nev; e += NT / 32) {
    if (a.hel_out) {
      const int k = warp_inverse_cdf<(P::NHEL + 31) / 32>(ng, a.hel_rnd[e0 + e], lane,
                                                          [&](int i) { return sm2[e * ng + i]; });
      if (lane == 0) a.hel_out[e0 + e] = k < 0 ? -1 : good[k];
    }
    if (a.col_out) {
      R x = R(0);
      if (lane < NC)
        for (int k = 0; k < ng; ++k) x += wj[(e * ng + k) * NCP + lane];
      const double w = (double)x;
      const int c = warp_inverse_cdf<1>(NC, a.col_rnd[e0 + e], lane, [&](int) { return w; });
      if (lane == 0) a.col_out[e0 + e] = c;
    }
  }
}

// Record of one event's current variants and momentum table in global memory
// (the kernel-split variant: the first kernel writes them, the second reads
// them back into shared memory): HS_NSLOT slots of 16-byte planes, then the
// momentum table K[NMOM][4] in the working precision.
template <class P, class R>
struct HsRecord {
  static constexpr int CUR = P::HS_NSLOT * Slots<R, 1>::NPL;
  static_assert((P::NMOM * 4 * sizeof(R)) % 16 == 0, "momentum table in 16-byte words");
  static constexpr int KW = (int)(P::NMOM * 4 * sizeof(R) / 16);
  static constexpr int WORDS = CUR + KW;
};

// Where a group's momenta come from: the momentum buffer (mg_sigmakin), the
// kernel-split records (current variants and momentum tables instead), or
// RAMBO inside the kernel (mg_sigmakin_rambo, mg_sigmakin_seeded).
constexpr int kSrcMomenta = 0, kSrcRecords = 1, kSrcRambo = 2;

// One event's RAMBO inside a SIGMAKIN kernel: the uniforms as the RAMBO kernel
// reads or draws them, the same forward code (rambo_forward), the momenta of
// all legs into out[leg][mu] (shared memory, FP64; the beams as the RAMBO
// kernel writes them) and the weight into wgt.  Not inlined, so that RAMBO's
// many FP64 temporaries do not raise the register count of the calling
// kernel (the call runs on a few lanes, once per event).
template <int NF>
__device__ __noinline__ void rambo_event_fused(const double* __restrict__ rnd, int64_t nevt, int64_t i, uint64_t key,
                                               int64_t first_event, double ecm, const RamboSetup& st, double* out,
                                               double* __restrict__ wgt) {
  double r[4 * NF];
  if (rnd) {
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) r[k] = rnd[(int64_t)k * nevt + i];
  } else {
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) r[k] = sm64_uniform(key, first_event + i, k);
  }
  RamboState<NF> z;
  rambo_forward<NF>(r, ecm, st, z);
  const double h = 0.5 * ecm;
  out[0] = h; out[1] = 0.0; out[2] = 0.0; out[3] = h;
  out[4] = h; out[5] = 0.0; out[6] = 0.0; out[7] = -h;
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) out[(2 + f) * 4 + mu] = z.k[f][mu];
  wgt[i] = z.w;
}

// The helicity-shared program for the events [first, last) of the batch.
// SRC == kSrcRecords: phases 1-2 (momenta, tables, current variants) are
// replaced by a copy of the events' records from `rec` (one record per event,
// event first - first at rec[0]).
template <class P, class R, int CS, int SRC>
__device__ __forceinline__ void hs_sigmakin_body(const SigArgs& a, const Couplings<R>& cp, int64_t first, int64_t last,
                                                 const uint4* __restrict__ rec, const RamboArgs* ra = nullptr) {
  using C = HsCfg<P, R>;
  using L = HsLayout<P, R, CS>;
  constexpr bool FROM_RECORDS = SRC == kSrcRecords;
  static_assert(!(FROM_RECORDS && L::TC), "the kernel-split variant sums colours on CUDA cores");
  constexpr int NT = C::NT, NC = P::NCOLOR;
  extern __shared__ __align__(1024) unsigned char smem[];
  int* good = reinterpret_cast<int*>(smem + L::o_good);
  int* misc = reinterpret_cast<int*>(smem + L::o_misc);
  double* sm2 = reinterpret_cast<double*>(smem + L::o_m2);
  uint8_t* vtab = reinterpret_cast<uint8_t*>(smem + L::o_vt);
  // per event: HS_NSLOT current slots, HS_XCAP amputated slots (16-byte planes)
  uint4* curs = reinterpret_cast<uint4*>(smem + L::o_cur);
  uint4* xbufs = reinterpret_cast<uint4*>(smem + L::o_x);
  constexpr int CUR_EV = L::CUR_EV, X_EV = L::X_EV;
  const int tid = threadIdx.x, lane = tid & 31;
  hs_setup_words<P, R, L>(smem, a.pp);
  // vt[S][ihel]: variant index of leg set S for helicity ihel (generated table)
  static_assert(((1 << P::NPAR) * P::NHEL) % 16 == 0, "variant table copied in 16-byte words");
  for (int i = tid; i < (1 << P::NPAR) * P::NHEL / 16; i += NT)
    reinterpret_cast<uint4*>(vtab)[i] = reinterpret_cast<const uint4*>(P::hs_variants())[i];
  // good helicities: every warp ballots the mask itself (32 helicities per
  // word), so the events and their momenta are known before any barrier;
  // good[] in helicity order (read only after later barriers)
  static_assert(P::NHEL <= 64 && NT >= P::NHEL, "helicity ballot layout");
  const unsigned w0 = __ballot_sync(0xffffffffu, lane < P::NHEL && a.mask[lane] != 0);
  const unsigned w1 = P::NHEL > 32 ? __ballot_sync(0xffffffffu, lane + 32 < P::NHEL && a.mask[lane + 32] != 0) : 0u;
  if (tid < P::NHEL) {
    const unsigned w = tid < 32 ? w0 : w1, bit = 1u << (tid & 31);
    if (w & bit) good[__popc(w & (bit - 1u)) + (tid >= 32 ? __popc(w0) : 0)] = tid;
  }
  const int ng = __popc(w0) + __popc(w1);
  const int ev = ng > 0 ? min(L::EVCAP, NT / ng) : C::EVMIN;
  // groups of ev events, g = blockIdx.x, blockIdx.x + gridDim.x, ...: one
  // group per CTA for a grid of all groups, several for a persistent grid
  const int ngrp = (int)((last - first + ev - 1) / ev);
  if ((int)blockIdx.x >= ngrp) return;
  if (ng == 0) {
    for (int g = blockIdx.x; g < ngrp; g += gridDim.x) {
      const int64_t e0 = first + (int64_t)g * ev;
      if (tid < (int)min((int64_t)ev, last - e0)) {
        a.me[e0 + tid] = 0.0;
        if (a.hel_out) a.hel_out[e0 + tid] = -1;
        if (a.col_out) a.col_out[e0 + tid] = -1;
        if constexpr (SRC == kSrcRambo)  // the weight all the same
          rambo_event_fused<P::NPAR - 2>(ra->rnd, a.nevt, e0 + tid, ra->key, ra->first_event, ra->ecm, ra->st,
                                         reinterpret_cast<double*>(smem + L::o_ps) + tid * P::NPAR * 4, ra->wgt);
      }
    }
    return;
  }
  uint32_t tmem = 0, mbar = 0;
  if constexpr (L::TC) {
    if (tid < 32) tc::tmem_alloc(tc::smem_addr(misc + 1), L::TMEM_COLS);
    mbar = tc::smem_addr(misc + 4);
    if (tid == 0) tc::mbar_init(mbar, 1);
    tc::fence_async_shared();
    tc::fence_before_sync();
  }
  const R* Kall = reinterpret_cast<const R*>(smem + L::o_K);
  const HsItem* items = P::hs_items();
  if constexpr (SRC == kSrcMomenta) {
    // the first group's momenta; later groups' arrive by prefetch
    const int64_t e0 = first + (int64_t)blockIdx.x * ev;
    hs_load_momenta<P, R, L>(smem, a.mom, a.nevt, e0, (int)min((int64_t)ev, last - e0));
  } else if constexpr (SRC == kSrcRambo) {
    // the first group's RAMBO, one lane per event, into the staging buffer
    const int64_t e0 = first + (int64_t)blockIdx.x * ev;
    const int nev0 = (int)min((int64_t)ev, last - e0);
    if (tid < nev0)
      rambo_event_fused<P::NPAR - 2>(ra->rnd, a.nevt, e0 + tid, ra->key, ra->first_event, ra->ecm, ra->st,
                                     reinterpret_cast<double*>(smem + L::o_ps) + tid * P::NPAR * 4, ra->wgt);
    __syncthreads();
    hs_convert_momenta<P, R, L>(smem, nev0);
  }
  __syncthreads();
  if constexpr (L::TC) {
    tc::fence_after_sync();
    tmem = static_cast<uint32_t>(misc[1]);
  }
#pragma unroll 1
  for (int g = blockIdx.x; g < ngrp; g += gridDim.x) {
    // e0 and nev are formed again after the contractions (fewer live registers)
    const int nev = (int)min((int64_t)ev, last - (first + (int64_t)g * ev));
    const HsGroup grp = hs_group<NT>(L::TC || !MG_HS_EVENT_SYNC, ng, ev, nev);
    if constexpr (FROM_RECORDS) {
      // 1-2. the events' current variants and momentum tables from their records
      using RC = HsRecord<P, R>;
      const uint4* in = rec + (int64_t)g * ev * RC::WORDS;
      uint4* ks = reinterpret_cast<uint4*>(smem + L::o_K);
      for (int t = tid; t < nev * RC::WORDS; t += NT) {
        const int e = t / RC::WORDS, w = t - e * RC::WORDS;
        const uint4 v = __ldcs(in + t);  // read once: streaming
        if (w < RC::CUR) curs[e * CUR_EV + w] = v;
        else ks[e * (L::KEV * (int)sizeof(R) / 16) + (w - RC::CUR)] = v;
      }
      __syncthreads();
    } else {
      // the next group's momenta: copied during this group's phases 1-2 and
      // converted after the last current level (p is free once the tables are built)
      const int gn = g + gridDim.x;
      const int64_t e0n = first + (int64_t)gn * ev;
      const int nevn = gn < ngrp ? (int)min((int64_t)ev, last - e0n) : 0;
      if constexpr (SRC == kSrcRambo) {
        // the next group's RAMBO on the last lanes, which the tables phase
        // leaves idle when it has fewer items than threads
        const int u = NT - 1 - tid;
        if (u < nevn)
          rambo_event_fused<P::NPAR - 2>(ra->rnd, a.nevt, e0n + u, ra->key, ra->first_event, ra->ecm, ra->st,
                                         reinterpret_cast<double*>(smem + L::o_ps) + u * P::NPAR * 4, ra->wgt);
      } else {
        if (nevn > 0) hs_prefetch_momenta<P, L>(smem, a.mom, a.nevt, e0n, nevn);
      }
      // 1. per-event tables (the momenta are in p)
      hs_tables<P, R, L, CUR_EV, L::KEV>(smem, a.pp, grp, curs, cp);
      const cx<R>* prall = reinterpret_cast<const cx<R>*>(smem + L::o_pr);
      // 2. current variants, level by level (level 0, the external wavefunctions,
      //    came with phase 1); consecutive threads take one item for each event (hs_item_of)
#pragma unroll
      for (int l = 1; l < P::HS_NLEVEL; ++l) {
        const int i0 = P::hs_level(l), ni = P::hs_level(l + 1) - i0, n = ni * grp.nev;
        for (int t = grp.j; t < n; t += grp.tpg) {
          const int ii = hs_item_of<L>(t, grp.nev), e = grp.ev0 + t - ii * grp.nev;
          const HsItem it = items[i0 + ii];
          hs_item<P, R>(it, Slots<R, P::HS_NSLOT>{curs + e * CUR_EV}, Kall + e * L::KEV, prall + e * P::NPROP,
                        cp);
        }
        if (l == P::HS_NLEVEL - 1) {
          cp_async_wait_all();
          __syncthreads();
          if (nevn > 0) hs_convert_momenta<P, R, L>(smem, nevn);
        } else {
          grp.sync();
        }
      }
    }
    // 3. amputated currents chunk by chunk into two alternating buffers: in
    //    interval c every thread first builds its share of chunk c, then
    //    contracts chunk c - 1 for its (event, helicity) (J in registers), so the
    //    latency of the item work hides behind other warps' contractions
    const bool active = tid < nev * ng;
    const int e = active ? tid / ng : 0;
    const int ih = good[active ? tid - e * ng : 0];
    constexpr int XBUF = L::EVCAP * X_EV;  // one chunk buffer, all events
    cx<R> J[NC];
#pragma unroll
    for (int s = 0; s < NC; ++s) J[s] = cx<R>(R(0), R(0));
#pragma unroll 1
    for (int c = 0; c <= P::HS_NXCHUNK; ++c) {
      if (c < P::HS_NXCHUNK) {
        uint4* xb = xbufs + (P::HS_XBUFS == 2 ? (c & 1) * XBUF : 0);
        const int i0 = P::hs_xitem(c), ni = P::hs_xitem(c + 1) - i0, n = ni * grp.nev;
        for (int t = grp.j; t < n; t += grp.tpg) {
          const int ii = hs_item_of<L>(t, grp.nev), ex = grp.ev0 + t - ii * grp.nev;
          const HsItem it = items[i0 + ii];
          hs_xitem<P, R>(it, Slots<R, P::HS_NSLOT>{curs + ex * CUR_EV}, Slots<R, P::HS_XCAP>{xb + ex * X_EV},
                         Kall + ex * L::KEV, cp);
        }
      }
      if (c > 0) {
        const uint4* xb = xbufs + (P::HS_XBUFS == 2 ? ((c - 1) & 1) * XBUF : 0);
        P::template hs_contract<R>(c - 1, Slots<R, P::HS_NSLOT>{curs + e * CUR_EV},
                                   Slots<R, P::HS_XCAP>{const_cast<uint4*>(xb) + e * X_EV}, vtab + ih, J);
      }
      if (c < P::HS_NXCHUNK) grp.sync();
    }
    // 4. colour sum and helicity sum
    double m2;
    if constexpr (L::TC) {
      __syncthreads();  // the A tiles overwrite the current variants
      m2 = (double)colour_sum_tc_regs<P, L>(smem, J, tmem, mbar);
    } else {
      m2 = (double)colour_sum_sym<P, R>(J);
    }
    sm2[tid] = active ? m2 : 0.0;
    if constexpr (L::TC) tc::fence_before_sync();
    grp.sync();
    const int64_t e0 = first + (int64_t)g * ev;
    // fixed-order FP64 helicity sum per event: eight lanes per event each add
    // every eighth helicity in order, then a butterfly over the eight lanes
    // (addition commutes, so every lane ends with the same bits); sm2 is next
    // written at the end of the next group, after several barriers
    for (int b = 0; b < grp.nev * 8; b += grp.tpg) {
      const int t = b + grp.j, eh = grp.ev0 + (t >> 3), q = t & 7;
      double sum = 0.0;
      if (t < grp.nev * 8) {
#pragma unroll
        for (int i = 0; i < (P::NHEL + 7) / 8; ++i)
          if (q + 8 * i < ng) sum += sm2[eh * ng + q + 8 * i];
      }
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      sum += __shfl_xor_sync(0xffffffffu, sum, 4);
      if (t < grp.nev * 8 && q == 0) a.me[e0 + eh] = sum * P::NORM;
    }
    // 5. helicity and colour-flow choices (batched entry point), once every
    //    group of the CTA is done with the union region; the closing barrier
    //    keeps the next group's currents out of it until the choices are made
    if (a.hel_out || a.col_out) {
      __syncthreads();
      if (a.col_out) {
        R* wj = reinterpret_cast<R*>(smem + L::o_U) + tid * HsChoice<P, R>::NCP;  // the union is dead here
#pragma unroll
        for (int s = 0; s < NC; ++s) wj[s] = active ? J[s].re * J[s].re + J[s].im * J[s].im : R(0);
        __syncthreads();
      }
      hs_choices<P, R, L>(smem, a, e0, nev, ng, good, sm2);
      __syncthreads();
    }
  }
  if constexpr (L::TC) {
    if (tid < 32) {
      tc::fence_after_sync();
      tc::tmem_dealloc(tmem, L::TMEM_COLS);
    }
  }
}

template <class P, class R, int CS>
__global__ void __launch_bounds__(HsCfg<P, R>::NT, HsCfg<P, R>::CTAS) sigmakin_hs_kernel(SigArgs a, Couplings<R> cp) {
  hs_sigmakin_body<P, R, CS, kSrcMomenta>(a, cp, 0, a.nevt, nullptr);
}

// RAMBO and SIGMAKIN in one kernel: no momentum buffer in HBM
template <class P, class R, int CS>
__global__ void __launch_bounds__(HsCfg<P, R>::NT, HsCfg<P, R>::CTAS)
    sigmakin_hs_rambo_kernel(SigArgs a, Couplings<R> cp, RamboArgs ra) {
  hs_sigmakin_body<P, R, CS, kSrcRambo>(a, cp, 0, a.nevt, nullptr, &ra);
}

}  // namespace mg
