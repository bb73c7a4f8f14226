// SIGMAKIN with helicity-shared currents (the default kernel of both modes).
//
// Same result as the straight-line kernel (sigmakin.cuh) — the same Feynman
// diagrams, colour flows and colour matrix (Sec. 2) — organised for GB300:
//   * an off-shell current over legs S depends only on the helicities of S,
//     so each current is computed once per event for each of its 2^|S|
//     helicity variants (not once per event helicity), into shared memory;
//   * every diagram's amplitude is formed at the vertex (chosen by the
//     generator) that needs the cheapest set of such currents;
//   * both the current items and the amplitude list are tables walked by
//     short loops, so the program is a few hundred instructions that stay in
//     the instruction cache (the unrolled gg -> t t~ g g program streams
//     ~30k instructions per helicity from L2).
// CTA of NT threads = EV events x ngood helicities.  Phases:
//   1. per-event momenta, momentum sums and FP64 propagator factors (as SIGMAKIN);
//   2. current variants, level by level (a level only reads earlier levels);
//   3. one thread per (event, helicity): loop over the amplitudes, operands from
//      shared memory (re-used while consecutive amplitudes share them), each
//      amplitude added into its colour flows J (shared memory);
//   4. colour sum (CUDA cores, or tcgen05 as in sigmakin.cuh) and the
//      fixed-order FP64 helicity sum.
#pragma once
#include "sigmakin.cuh"

namespace mg {

template <class P, class R>
struct HsCfg {
  using C = SigCfg<P>;
  static constexpr int NT = C::NT;
  static constexpr size_t CUR_BUDGET = 48 * 1024 * (sizeof(R) / 4);  // shared memory for current variants
  static constexpr int FIT = (int)(CUR_BUDGET / (P::HS_NSLOT * sizeof(W4<R>)));
  static constexpr int EVCAP = (FIT < C::EVCAP ? (FIT > C::EVMIN ? FIT : C::EVMIN) : C::EVCAP);
};

template <class P, class R, int CS>
struct HsLayout {
  using C = SigCfg<P>;
  using H = HsCfg<P, R>;
  static constexpr int EVCAP = H::EVCAP;
  static constexpr bool TC = CS == CS_TC;
  static constexpr size_t o_momtab = 0;
  static constexpr size_t o_proptab = align_up(o_momtab + 12 * P::NMOM, 16);
  static constexpr size_t o_good = align_up(o_proptab + 8 * P::NPROP, 16);
  static constexpr size_t o_misc = align_up(o_good + 4 * P::NHEL, 16);
  static constexpr size_t o_p = align_up(o_misc + 32, 16);
  static constexpr size_t o_K = align_up(o_p + 8 * EVCAP * P::NPAR * 4, 16);
  static constexpr size_t o_pr = align_up(o_K + sizeof(R) * EVCAP * P::NMOM * 4, 16);
  static constexpr size_t o_m2 = align_up(o_pr + 2 * sizeof(R) * EVCAP * P::NPROP, 16);
  static constexpr size_t o_slot = align_up(o_m2 + 8 * C::NT, 16);
  static constexpr size_t o_cur = align_up(o_slot + 2 * P::HS_NCUR * P::NHEL, 128);
  static constexpr size_t o_J = align_up(o_cur + sizeof(W4<R>) * EVCAP * P::HS_NSLOT, 128);
  static constexpr size_t o_A = align_up(o_J + 2 * sizeof(R) * P::NCOLOR * C::NT, 1024);
  static constexpr size_t tileA = 128 * C::KP * 2;
  static constexpr size_t o_B = o_A + (TC ? 3 * 2 * C::MBLK * tileA : 0);
  static constexpr size_t bytes = o_B + (TC ? C::NP * C::KP * 2 : 0);
  static constexpr uint32_t TMEM_COLS = C::MBLK * 2 * C::NP;
  static_assert(bytes <= 232448, "shared memory per CTA above the 227 KB limit");
};

// one current variant
template <class P, class R>
__device__ __forceinline__ void hs_item(const HsItem& it, W4<R>* cur, const R* K, const cx<R>* pr,
                                        const Couplings<R>& cp) {
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
    default:
      o = vvvv_comb(cur[it.in[0]], vdot(cur[it.in[1]], cur[it.in[2]]), cur[it.in[3]],
                    vdot(cur[it.in[4]], cur[it.in[5]]), mul_mi(cp.gs2 * pr[it.prop]));
  }
  cur[it.out] = o;
}

template <class P, class R, int CS>
__global__ void __launch_bounds__(SigCfg<P>::NT, 1) sigmakin_hs_kernel(SigArgs a, Couplings<R> cp) {
  using C = SigCfg<P>;
  using L = HsLayout<P, R, CS>;
  constexpr int NT = C::NT, NC = P::NCOLOR;
  extern __shared__ __align__(1024) unsigned char smem[];
  int* good = reinterpret_cast<int*>(smem + L::o_good);
  int* misc = reinterpret_cast<int*>(smem + L::o_misc);
  double* sm2 = reinterpret_cast<double*>(smem + L::o_m2);
  uint16_t* slots = reinterpret_cast<uint16_t*>(smem + L::o_slot);
  W4<R>* curs = reinterpret_cast<W4<R>*>(smem + L::o_cur);
  R* Js = reinterpret_cast<R*>(smem + L::o_J);
  const int tid = threadIdx.x;
  load_tables<P, L>(smem);
  if (tid == 0) {
    int n = 0;
    for (int h = 0; h < P::NHEL; ++h)
      if (a.mask[h]) good[n++] = h;
    misc[0] = n;
  }
  {
    const uint16_t* src = P::hs_slots();
    for (int i = tid; i < P::HS_NCUR * P::NHEL; i += NT) slots[i] = src[i];
  }
  __syncthreads();
  const int ng = misc[0];
  const int ev = ng > 0 ? min(L::EVCAP, NT / ng) : C::EVMIN;
  const int64_t e0 = (int64_t)blockIdx.x * ev;
  if (e0 >= a.nevt) return;
  const int nev = (int)min((int64_t)ev, a.nevt - e0);
  if (ng == 0) {
    if (tid < nev) a.me[e0 + tid] = 0.0;
    return;
  }
  uint32_t tmem = 0, mbar = 0;
  if constexpr (L::TC) {
    if (tid < 32) tc::tmem_alloc(tc::smem_addr(misc + 1), L::TMEM_COLS);
    mbar = tc::smem_addr(misc + 4);
    if (tid == 0) tc::mbar_init(mbar, 1);
    const uint4* src = reinterpret_cast<const uint4*>(P::colour_bf16_image());
    uint4* dst = reinterpret_cast<uint4*>(smem + L::o_B);
    for (int i = tid; i < C::NP * C::KP * 2 / 16; i += NT) dst[i] = src[i];
    tc::fence_async_shared();
    tc::fence_before_sync();
  }
  // 1. momenta and per-event tables
  event_tables<P, R, L>(smem, a, e0, nev);
  if constexpr (L::TC) {
    tc::fence_after_sync();
    tmem = static_cast<uint32_t>(misc[1]);
  }
  const R* Kall = reinterpret_cast<const R*>(smem + L::o_K);
  const cx<R>* prall = reinterpret_cast<const cx<R>*>(smem + L::o_pr);
  // 2. current variants, level by level; consecutive threads take the same
  //    item for consecutive events
  const HsItem* items = P::hs_items();
#pragma unroll
  for (int l = 0; l < P::HS_NLEVEL; ++l) {
    const int i0 = P::hs_level(l), n = (P::hs_level(l + 1) - i0) * nev;
    for (int t = tid; t < n; t += NT) {
      const int e = t % nev;
      const HsItem it = items[i0 + t / nev];
      hs_item<P, R>(it, curs + e * P::HS_NSLOT, Kall + e * P::NMOM * 4, prall + e * P::NPROP, cp);
    }
    __syncthreads();
  }
  // 3. amplitudes of this thread's (event, helicity), J in registers
  const bool active = tid < nev * ng;
  const int e = active ? tid / ng : 0;
  const int ih = good[active ? tid - e * ng : 0];
  const W4<R>* cur = curs + e * P::HS_NSLOT;
  const R* K = Kall + e * P::NMOM * 4;
  const uint16_t* sl = slots + ih;
  cx<R> J[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) J[s] = cx<R>(R(0), R(0));
  P::template hs_amplitudes<R>(cur, sl, K, cp, J);
  R* Jr = Js + tid;
  R* Ji = Js + NC * NT + tid;
#pragma unroll
  for (int s = 0; s < NC; ++s) { Jr[s * NT] = J[s].re; Ji[s * NT] = J[s].im; }
  // 4. colour sum and helicity sum
  double m2;
  if constexpr (L::TC) {
    __syncthreads();
    m2 = (double)colour_sum_tc<P, L>(smem, Js, tmem, mbar);
  } else {
    m2 = (double)colour_sum_simt<P, R>([&](int s) { return J[s].re; }, [&](int s) { return J[s].im; });
  }
  sm2[tid] = active ? m2 : 0.0;
  if constexpr (L::TC) tc::fence_before_sync();
  __syncthreads();
  if constexpr (L::TC) {
    if (tid < 32) {
      tc::fence_after_sync();
      tc::tmem_dealloc(tmem, L::TMEM_COLS);
    }
  }
  if (tid < nev) {
    double sum = 0.0;
    for (int k = 0; k < ng; ++k) sum += sm2[tid * ng + k];
    a.me[e0 + tid] = sum * P::NORM;
  }
}

}  // namespace mg
