// Gradient d me / d rnd with the helicity-shared program (not in the paper):
// the forward pass of sigmakin_hs.cuh with every variant slot kept in shared
// memory, then its adjoint.  Three launches: RAMBO (one thread per event,
// FP64) leaves the final-state momenta in the gradient buffer; the main kernel
// runs, for the CTA's events:
//   1. the momenta from that buffer;
//   2. tables, current variants, amputated currents, contractions, colour sum
//      (as SIGMAKIN, one chunk of amputated currents);
//   3. per (event, helicity): Jb = dL/dJ from the colour sum,
//      Jb_s = (dL/dme) NORM 2 (C J)_s / CDEN, then the adjoint contractions in
//      two passes: into the shared adjoint slots of the operands (they read
//      the amputated currents X), then into the amputated currents' adjoints,
//      which take X's storage (they read only the operands);
//   4. the amputated currents' and currents' adjoints, level by level in
//      reverse, into their inputs, the momentum table and the propagators;
//   5. external wavefunctions (forward-mode momentum Jacobians) and the
//      propagators into the momenta; the momentum table into the legs;
//   6. dL/d(final momenta) back into the buffer;
// then the RAMBO adjoint (one thread per event, FP64) -> dL/d rnd; rows RAMBO
// does not consume get 0.  Many helicities share a variant: the adjoint
// contractions sum them with warp shuffles (shared-memory atomics when the
// helicities of an event do not fill whole warps); the item adjoints of an
// event run on one warp, whose lanes with the same destination sum through a
// shared-memory staging area before one lane adds (no atomics); the external
// and propagator adjoints add atomically, so the last bits of a result may
// vary between runs.
// Adjoint convention of helas_adj.cuh: zb = dL/dRe z + i dL/dIm z.
#pragma once
#include "grad.cuh"
#include "sigmakin_hs.cuh"

namespace mg {

// events per CTA: small FP32 CTAs, several per SM, overlap each other's
// latency-bound phases; the FP64 kernel prefers larger ones (measured)
#ifndef MG_HSG_EV
#define MG_HSG_EV 2
#endif
#ifndef MG_HSG_EV64
#define MG_HSG_EV64 8
#endif

template <class P, class R>
struct HsGradCfg {
  static constexpr int EVW = sizeof(R) == 4 ? MG_HSG_EV : MG_HSG_EV64;
  // at least one whole warp (the adjoint's warp sums shuffle across all 32 lanes)
  static constexpr int NT = EVW * P::NHEL >= 32 ? EVW * P::NHEL : 32;
  static constexpr int EVMIN = NT / P::NHEL;
  static constexpr int EVCAP = EVMIN;
  static_assert(P::HS_NXCHUNK == 1, "the adjoint keeps every amputated current: one chunk");
};

template <class P, class R>
struct HsGradLayout {
  using H = HsGradCfg<P, R>;
  static constexpr int NT = H::NT, EVCAP = H::EVCAP, NF = P::NFINAL;
  static constexpr size_t W = sizeof(W4<R>);
  static constexpr size_t o_proptab = 0;
  static constexpr size_t o_md = align_up(o_proptab + 8 * P::NPROP, 16);  // momentum-entry descriptors (int4)
  static constexpr size_t o_good = align_up(o_md + 16 * P::NMOM, 16);
  static constexpr size_t o_misc = align_up(o_good + 4 * P::NHEL, 16);
  static constexpr size_t o_mconst = align_up(o_misc + 32, 16);
  static constexpr size_t o_p = align_up(o_mconst + 32, 16);  // [EV][NPAR][4]: double, or float2 (hi, lo) in FP32
  static constexpr size_t o_pb = align_up(o_p + 8 * EVCAP * P::NPAR * 4, 16);          // double [EV][NPAR][4]
  static constexpr size_t o_K = align_up(o_pb + 8 * EVCAP * P::NPAR * 4, 16);          // R [EV][NMOM][4]
  static constexpr size_t o_Kb = align_up(o_K + sizeof(R) * EVCAP * P::NMOM * 4, 16);  // R [EV][NMOM][4]
  static constexpr size_t o_pr = align_up(o_Kb + sizeof(R) * EVCAP * P::NMOM * 4, 16);  // cx<R> [EV][NPROP]
  static constexpr size_t o_prb = align_up(o_pr + 2 * sizeof(R) * EVCAP * P::NPROP, 16);
  // R [NT]: each thread's |M_h|^2, formed in R (stored exactly; summed in FP64)
  static constexpr size_t o_m2 = align_up(o_prb + 2 * sizeof(R) * EVCAP * P::NPROP, 16);
  static constexpr size_t o_vt = align_up(o_m2 + sizeof(R) * NT, 16);
  static constexpr size_t o_cur = align_up(o_vt + (size_t(1) << P::NPAR) * P::NHEL, 128);
  static constexpr size_t o_curb = o_cur + W * EVCAP * P::HS_NSLOT;
  // the amputated currents X, then (second pass of the contraction adjoints)
  // their adjoints Xb in the same storage
  static constexpr size_t o_x = o_curb + W * EVCAP * P::HS_NSLOT;
  // staging of the item adjoints' group sums, one W4 per thread
  static constexpr size_t o_stage = o_x + W * EVCAP * P::HS_XCAP;
  static constexpr size_t bytes = o_stage + W * NT;
  static_assert(bytes <= 232448, "shared memory per CTA above the 227 KB limit");
};

template <class R>
__device__ __forceinline__ void atomic_add4(R* d, const R* v) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) atomicAdd(d + mu, v[mu]);
}
template <class R>
__device__ __forceinline__ void atomic_addc(cx<R>* d, cx<R> v) {
  atomicAdd(&d->re, v.re);
  atomicAdd(&d->im, v.im);
}

// Warp-aggregated adds for the item adjoints: the lanes of a warp that add into
// the same destination (same key: its shared-memory address) form a group, and
// only the lowest lane of each group adds, the group's values summed in lane
// order (its own first), so no two lanes of a warp write one address.  The
// values pass through the warp's staging area in shared memory (32 lanes x NV,
// at most 8 values of R per lane): every lane stores its values and each
// leader reads its members' (a group of n lanes costs its leader n - 1 reads,
// not n - 1 rounds of warp-wide shuffles).  The lanes taking part are the ones
// executing together (__activemask), and every collective below runs on all
// of them.
template <int NV, class R>
__device__ __forceinline__ bool warp_group_sum(unsigned key, R* v, R* stage) {
  static_assert(NV <= 8, "staging holds 8 values per lane");
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  const unsigned g = __match_any_sync(act, key);
  if (!__any_sync(act, g != (1u << lane))) return true;  // every lane alone: no sums
  R* mine = stage + 8 * lane;
  if constexpr ((NV * sizeof(R)) % 16 == 0) {
#pragma unroll
    for (int i = 0; i < (int)(NV * sizeof(R) / 16); ++i)
      reinterpret_cast<uint4*>(mine)[i] = reinterpret_cast<const uint4*>(v)[i];
  } else {
#pragma unroll
    for (int i = 0; i < NV; ++i) mine[i] = v[i];
  }
  __syncwarp(act);
  const bool leader = lane == __ffs(g) - 1;
  if (leader) {
    unsigned others = g & ~(1u << lane);
    while (others) {
      const int src = __ffs(others) - 1;
      others &= others - 1;
      const R* o = stage + 8 * src;
      if constexpr ((NV * sizeof(R)) % 16 == 0) {
        R t[NV];
#pragma unroll
        for (int i = 0; i < (int)(NV * sizeof(R) / 16); ++i)
          reinterpret_cast<uint4*>(t)[i] = reinterpret_cast<const uint4*>(o)[i];
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += t[i];
      } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += o[i];
      }
    }
  }
  __syncwarp(act);
  return leader;
}
__device__ __forceinline__ unsigned smem_key(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Adds into destinations that only the calling warp writes during the phase
// (each event's item adjoints run on one warp): the group's lowest lane adds
// the group sum with a plain read-modify-write; the caller separates rounds of
// items with __syncwarp.
template <class R>
__device__ __forceinline__ void own_add4(R* d, const R* v, R* stage) {
  alignas(16) R t[4] = {v[0], v[1], v[2], v[3]};
  if (warp_group_sum<4>(smem_key(d), t, stage)) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) d[mu] += t[mu];
  }
}
template <class R>
__device__ __forceinline__ void own_addc(cx<R>* d, cx<R> v, R* stage) {
  alignas(16) R t[2] = {v.re, v.im};
  if (warp_group_sum<2>(smem_key(d), t, stage)) *d = cx<R>(d->re + t[0], d->im + t[1]);
}
template <class R, int N>
__device__ __forceinline__ void own_slot_add(const Slots<R, N>& s, int i, const W4<R>& w, R* stage) {
  alignas(16) R t[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    t[2 * k] = w.w[k].re;
    t[2 * k + 1] = w.w[k].im;
  }
  if (warp_group_sum<8>(smem_key(s.p + i), t, stage)) {
    W4<R> o = s[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) o.w[k] = cx<R>(o.w[k].re + t[2 * k], o.w[k].im + t[2 * k + 1]);
    s.set(i, o);
  }
}

// adjoint of one current variant (levels >= 1)
template <class P, class R>
__device__ __forceinline__ void hs_item_adj(const HsItem& it, const Slots<R, P::HS_NSLOT>& cur,
                                            const Slots<R, P::HS_NSLOT>& curb, const R* K, R* Kb, const cx<R>* pr,
                                            cx<R>* prb, const Couplings<R>& cp, R* stage) {
  const W4<R> ob = curb[it.out];
  W4<R> b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) b[k] = w4_zero<R>();
  R kb0[4] = {R(0), R(0), R(0), R(0)}, kb1[4] = {R(0), R(0), R(0), R(0)};
  cx<R> pb(R(0), R(0));
  int nin = 2, nk = 0;
  switch (it.type) {
    case 3:
      FFV1_2_adj(cur[it.in[0]], cur[it.in[1]], cp.gs, K + 4 * it.k0, cp.mt, pr[it.prop], ob, b[0], b[1], kb0, pb);
      nk = 1;
      break;
    case 4:
      FFV1_1_adj(cur[it.in[0]], cur[it.in[1]], cp.gs, K + 4 * it.k0, cp.mt, pr[it.prop], ob, b[0], b[1], kb0, pb);
      nk = 1;
      break;
    case 5:
      FFV1P0_3_adj(cur[it.in[0]], cur[it.in[1]], it.a ? cp.ee : cp.gs, pr[it.prop], ob, b[0], b[1], pb);
      break;
    case 7:
      VVV1P0_1_adj(cur[it.in[0]], cur[it.in[1]], K + 4 * it.k0, K + 4 * it.k1, cp.gs, pr[it.prop], ob, b[0], b[1],
                   kb0, kb1, pb);
      nk = 2;
      break;
    default: {  // four-gluon term X_0 (X_1 . W) - X_1 (X_0 . W), in = {X_0, X_1, W}
      const W4<R> x0 = cur[it.in[0]], x1 = cur[it.in[1]], w = cur[it.in[2]];
      vvvv_adj(x0, x1, w, x1, x0, w, cp.gs2, pr[it.prop], ob, b[0], b[1], b[2], b[1], b[0], b[2], pb);
      nin = 3;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < nin) own_slot_add(curb, it.in[k], b[k], stage);
  if (nk >= 1) own_add4(Kb + 4 * it.k0, kb0, stage);
  if (nk >= 2) own_add4(Kb + 4 * it.k1, kb1, stage);
  own_addc(prb + it.prop, pb, stage);
}

// adjoint of one amputated-current variant
template <class P, class R>
__device__ __forceinline__ void hs_xitem_adj(const HsItem& it, const Slots<R, P::HS_NSLOT>& cur,
                                             const Slots<R, P::HS_NSLOT>& curb, const Slots<R, P::HS_XCAP>& xbb,
                                             const R* K, R* Kb, const Couplings<R>& cp, R* stage) {
  const W4<R> ob = xbb[it.out];
  W4<R> b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) b[k] = w4_zero<R>();
  R kb0[4] = {R(0), R(0), R(0), R(0)}, kb1[4] = {R(0), R(0), R(0), R(0)};
  int nin = 2;
  bool mom = false;
  switch (it.type) {
    case 9: FFV1_2A_adj(cur[it.in[0]], cur[it.in[1]], cp.gs, ob, b[0], b[1]); break;
    case 10: FFV1_1A_adj(cur[it.in[0]], cur[it.in[1]], cp.gs, ob, b[0], b[1]); break;
    case 11: FFV1P0_3A_adj(cur[it.in[0]], cur[it.in[1]], it.a ? cp.ee : cp.gs, ob, b[0], b[1]); break;
    case 13:
      VVV1P0_1A_adj(cur[it.in[0]], cur[it.in[1]], K + 4 * it.k0, K + 4 * it.k1, cp.gs, ob, b[0], b[1], kb0, kb1);
      mom = true;
      break;
    default: {  // four-gluon term, as in hs_item_adj
      const W4<R> x0 = cur[it.in[0]], x1 = cur[it.in[1]], w = cur[it.in[2]];
      vvvv_comb_a_adj(x0, x1, w, x1, x0, w, cp.gs2, ob, b[0], b[1], b[2], b[1], b[0], b[2]);
      nin = 3;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < nin) own_slot_add(curb, it.in[k], b[k], stage);
  if (mom) {
    own_add4(Kb + 4 * it.k0, kb0, stage);
    own_add4(Kb + 4 * it.k1, kb1, stage);
  }
}

template <class P, class R>
__global__ void __launch_bounds__(HsGradCfg<P, R>::NT) sigmakin_hs_grad_kernel(GradArgs a, Couplings<R> cp) {
  using L = HsGradLayout<P, R>;
  constexpr int NT = L::NT, NC = P::NCOLOR, NF = P::NFINAL;
  constexpr int CUR_EV = P::HS_NSLOT * Slots<R, 1>::NPL, X_EV = P::HS_XCAP * Slots<R, 1>::NPL;
  extern __shared__ __align__(1024) unsigned char smem[];
  int* good = reinterpret_cast<int*>(smem + L::o_good);
  int* misc = reinterpret_cast<int*>(smem + L::o_misc);
  R* sm2 = reinterpret_cast<R*>(smem + L::o_m2);
  uint8_t* vtab = reinterpret_cast<uint8_t*>(smem + L::o_vt);
  auto pbs = reinterpret_cast<double(*)[P::NPAR][4]>(smem + L::o_pb);
  R* Kall = reinterpret_cast<R*>(smem + L::o_K);
  R* Kball = reinterpret_cast<R*>(smem + L::o_Kb);
  cx<R>* prall = reinterpret_cast<cx<R>*>(smem + L::o_pr);
  cx<R>* prball = reinterpret_cast<cx<R>*>(smem + L::o_prb);
  uint4* curs = reinterpret_cast<uint4*>(smem + L::o_cur);
  uint4* cursb = reinterpret_cast<uint4*>(smem + L::o_curb);
  uint4* xbufs = reinterpret_cast<uint4*>(smem + L::o_x);
  uint4* xbufsb = xbufs;  // Xb overwrites X in the second contraction-adjoint pass
  const int tid = threadIdx.x;
  // 0. tables, zeroed adjoints
  hs_setup_words<P, R, L>(smem, a.pp);
  static_assert(P::NHEL <= 64 && NT >= P::NHEL, "helicity ballot layout");
  const bool hgood = tid < P::NHEL && a.mask[tid] != 0;
  const unsigned hbal = __ballot_sync(0xffffffffu, hgood);
  if (tid < P::NHEL && (tid & 31) == 0) misc[2 + (tid >> 5)] = (int)hbal;
  for (int i = tid; i < (1 << P::NPAR) * P::NHEL / 16; i += NT)
    reinterpret_cast<uint4*>(vtab)[i] = reinterpret_cast<const uint4*>(P::hs_variants())[i];
  {
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < (int)((L::o_x - L::o_curb) / 16); i += NT) cursb[i] = z;
    for (int i = tid; i < (int)((L::o_pr - L::o_Kb) / 16); i += NT) reinterpret_cast<uint4*>(Kball)[i] = z;
    for (int i = tid; i < (int)((L::o_m2 - L::o_prb) / 16); i += NT) reinterpret_cast<uint4*>(prball)[i] = z;
    for (int i = tid; i < (int)((L::o_K - L::o_pb) / 16); i += NT) reinterpret_cast<uint4*>(&pbs[0][0][0])[i] = z;
  }
  __syncthreads();
  const unsigned w0 = (unsigned)misc[2], w1 = P::NHEL > 32 ? (unsigned)misc[3] : 0u;
  if (hgood) good[__popc(hbal & ((1u << (tid & 31)) - 1u)) + (tid >= 32 ? __popc(w0) : 0)] = tid;
  const int ng = __popc(w0) + __popc(w1);
  const int ev = ng > 0 ? min(L::EVCAP, NT / ng) : L::EVCAP;
  const int64_t e0 = (int64_t)blockIdx.x * ev;
  if (e0 >= a.nevt) return;
  const int nev = (int)min((int64_t)ev, a.nevt - e0);
  // 1. momenta: the beams, and the final states the RAMBO pass left in grad,
  //    in the layout of the forward kernel's p
  for (int t = tid; t < nev * P::NPAR * 4; t += NT) {
    const int e = t % nev, c = t / nev, l = c >> 2, mu = c & 3;
    const double h = 0.5 * a.ecm;
    const double x = l >= 2 ? a.grad[(int64_t)(c - 8) * a.nevt + e0 + e]
                            : (mu == 0 ? h : (mu == 3 ? (l == 0 ? h : -h) : 0.0));
    if constexpr (sizeof(R) == 4) {
      const dfl q = dfl_split(x);
      reinterpret_cast<float2*>(smem + L::o_p)[e * P::NPAR * 4 + c] = make_float2(q.hi, q.lo);
    } else {
      reinterpret_cast<double*>(smem + L::o_p)[e * P::NPAR * 4 + c] = x;
    }
  }
  __syncthreads();
  if (ng == 0) {
    for (int t = tid; t < nev * 4 * NF; t += NT) a.grad[(int64_t)(t / nev) * a.nevt + e0 + t % nev] = 0.0;
    if (tid < nev && a.me) a.me[e0 + tid] = 0.0;
    return;
  }
  // 2. forward: tables, currents, amputated currents, contractions, colour sum
  hs_tables<P, R, L>(smem, a.pp, HsGroup{0, NT, tid, 0, nev, 0}, curs, cp);
  const HsItem* items = P::hs_items();
#pragma unroll
  for (int l = 1; l < P::HS_NLEVEL; ++l) {
    const int i0 = P::hs_level(l), ni = P::hs_level(l + 1) - i0, n = ni * nev;
    for (int t = tid; t < n; t += NT) {  // item-major lanes, as the forward kernel
      const int ii = hs_item_of<L>(t, nev), e = t - ii * nev;
      const HsItem it = items[i0 + ii];
      hs_item<P, R>(it, Slots<R, P::HS_NSLOT>{curs + e * CUR_EV}, Kall + e * P::NMOM * 4, prall + e * P::NPROP, cp);
    }
    __syncthreads();
  }
  {
    const int i0 = P::hs_xitem(0), ni = P::hs_xitem(1) - i0, n = ni * nev;
    for (int t = tid; t < n; t += NT) {
      const int ii = hs_item_of<L>(t, nev), e = t - ii * nev;
      const HsItem it = items[i0 + ii];
      hs_xitem<P, R>(it, Slots<R, P::HS_NSLOT>{curs + e * CUR_EV}, Slots<R, P::HS_XCAP>{xbufs + e * X_EV},
                     Kall + e * P::NMOM * 4, cp);
    }
  }
  __syncthreads();
  const bool active = tid < nev * ng;
  const int e = active ? tid / ng : 0;
  const int ih = good[active ? tid - e * ng : 0];
  const Slots<R, P::HS_NSLOT> cur{curs + e * CUR_EV}, curb{cursb + e * CUR_EV};
  const Slots<R, P::HS_XCAP> xb{xbufs + e * X_EV}, xbb{xbufsb + e * X_EV};
  cx<R> J[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) J[s] = cx<R>(R(0), R(0));
  P::template hs_contract<R>(0, cur, xb, vtab + ih, J);
  const R m2 = colour_sum_sym<P, R>(J);
  sm2[tid] = active ? m2 : R(0);
  // 3. colour-sum adjoint, adjoint contractions (every thread takes part: the
  //    warp sums before the atomic adds need whole warps; idle threads add 0)
  {
    const double gl = active ? (a.gout ? a.gout[e0 + e] : 1.0) * P::NORM : 0.0;
    const R f = R(2.0 * gl / (double)P::CDEN);
    cx<R> Jb[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      cx<R> s(R(0), R(0));
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (P::cnum(i, j) != 0) s += R(P::cnum(i, j)) * J[j];
      Jb[i] = f * s;
    }
    // lanes = consecutive helicities of whole events when every helicity is good
    const bool full = ng == P::NHEL && (P::NHEL % 32 == 0 || 32 % P::NHEL == 0);
    // two passes, so that Xb needs no storage of its own: the operand adjoints
    // (they read X), then, with X dead and its storage zeroed, the amputated
    // currents' adjoints into that storage (they read the operands Y)
    P::template hs_contract_adj<1, R>(0, cur, xb, vtab + ih, Jb, curb, xbb, full, tid & 31, active);
    __syncthreads();
    for (int i = tid; i < L::EVCAP * X_EV; i += NT) xbufs[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    P::template hs_contract_adj<2, R>(0, cur, xb, vtab + ih, Jb, curb, xbb, full, tid & 31, active);
  }
  __syncthreads();
  // 4. amputated currents, then the current levels in reverse; the items of
  //    event ex run on warp ex % (NT / 32), so each event's adjoint slots have
  //    one writing warp (plain adds, rounds of 32 items separated by __syncwarp)
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int NW = NT / 32;
  R* const wstage = reinterpret_cast<R*>(smem + L::o_stage) + warp * 32 * 8;  // the warp's group-sum staging
  {
    const int i0 = P::hs_xitem(0), ni = P::hs_xitem(1) - i0;
    for (int ex = warp; ex < nev; ex += NW) {
      for (int r0 = 0; r0 < ni; r0 += 32) {
        if (r0 + lane < ni) {
          const HsItem it = items[i0 + r0 + lane];
          hs_xitem_adj<P, R>(it, Slots<R, P::HS_NSLOT>{curs + ex * CUR_EV},
                             Slots<R, P::HS_NSLOT>{cursb + ex * CUR_EV}, Slots<R, P::HS_XCAP>{xbufsb + ex * X_EV},
                             Kall + ex * P::NMOM * 4, Kball + ex * P::NMOM * 4, cp, wstage);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int l = P::HS_NLEVEL - 1; l >= 1; --l) {
    const int i0 = P::hs_level(l), ni = P::hs_level(l + 1) - i0;
    for (int ex = warp; ex < nev; ex += NW) {
      for (int r0 = 0; r0 < ni; r0 += 32) {
        if (r0 + lane < ni) {
          const HsItem it = items[i0 + r0 + lane];
          hs_item_adj<P, R>(it, Slots<R, P::HS_NSLOT>{curs + ex * CUR_EV}, Slots<R, P::HS_NSLOT>{cursb + ex * CUR_EV},
                            Kall + ex * P::NMOM * 4, Kball + ex * P::NMOM * 4, prall + ex * P::NPROP,
                            prball + ex * P::NPROP, cp, wstage);
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  // 5. external wavefunctions -> momenta; propagators -> momentum table
  {
    constexpr int NEXT = P::hs_level(1);
    const int2* prop_tab = reinterpret_cast<const int2*>(smem + L::o_proptab);
    for (int t = tid; t < nev * (NEXT + P::NPROP); t += NT) {
      if (t < nev * NEXT) {
        const int ex = t / NEXT;
        const HsItem it = items[t - ex * NEXT];
        const W4<R> ob = Slots<R, P::HS_NSLOT>{cursb + ex * CUR_EV}[it.out];
        R pk[4], pbk[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          const int ip = (ex * P::NPAR + it.a) * 4 + mu;
          if constexpr (sizeof(R) == 4) pk[mu] = reinterpret_cast<const float2*>(smem + L::o_p)[ip].x;
          else pk[mu] = reinterpret_cast<const double*>(smem + L::o_p)[ip];
        }
        external_adj<R>(it.type, pk, it.flag ? cp.mt : R(0), it.b, it.c, ob, pbk);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) atomicAdd(&pbs[ex][it.a][mu], (double)pbk[mu]);
      } else {
        const int t2 = t - nev * NEXT, ex = t2 / P::NPROP, j = t2 - ex * P::NPROP;
        const int2 m = prop_tab[j];
        R kb[4] = {R(0), R(0), R(0), R(0)};
        prop_adj(prall[ex * P::NPROP + j], m.y == 1, Kall + (ex * P::NMOM + m.x) * 4, prball[ex * P::NPROP + j], kb);
        atomic_add4(Kball + (ex * P::NMOM + m.x) * 4, kb);
      }
    }
  }
  __syncthreads();
  // 6. helicity sum (eight lanes per event in a fixed order, then a butterfly
  //    over the eight lanes, as the forward kernel); dL/d(final momenta) into
  //    grad for the RAMBO adjoint pass: one thread per (event, final leg,
  //    component) adds to the external wavefunctions' part the momentum-table
  //    entries that contain the leg (sign from the entry, four partial sums)
  for (int b = 0; b < nev * 8; b += NT) {
    const int t = b + tid, ex = t >> 3, q = t & 7;
    double sum = 0.0;
    if (t < nev * 8) {
#pragma unroll
      for (int i = 0; i < (P::NHEL + 7) / 8; ++i)
        if (q + 8 * i < ng) sum += sm2[ex * ng + q + 8 * i];
    }
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);
    sum += __shfl_xor_sync(0xffffffffu, sum, 2);
    sum += __shfl_xor_sync(0xffffffffu, sum, 4);
    if (t < nev * 8 && q == 0 && a.me) a.me[e0 + ex] = sum * P::NORM;
  }
  for (int t = tid; t < nev * 4 * NF; t += NT) {
    const int ex = t % nev, c = t / nev, l = 2 + (c >> 2), mu = c & 3;
    const R* Kb = Kball + ex * P::NMOM * 4;
    double acc[4] = {pbs[ex][l][mu], 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < P::NMOM; ++j) {
      if (!(P::mom(j, 1) >> l & 1)) continue;
      const bool neg = P::mom(j, 0) == 1 && (P::mom(j, 2) >> l & 1);
      const double kb = (double)Kb[4 * j + mu];
      acc[j & 3] += neg ? -kb : kb;
    }
    a.grad[(int64_t)c * a.nevt + e0 + ex] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
}

// three passes: RAMBO (final momenta into grad), the helicity-shared forward
// and adjoint (dL/d momenta into grad), the RAMBO adjoint (dL/d rnd into grad)
template <class P, class R>
cudaError_t launch_hs_grad_variant(const GradArgs& a, const Couplings<R>& cp, cudaStream_t s) {
  using L = HsGradLayout<P, R>;
  const int64_t grid = (a.nevt + HsGradCfg<P, R>::EVMIN - 1) / HsGradCfg<P, R>::EVMIN;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = launch_rambo_final(P::NFINAL, a.nevt, a.ecm, a.rnd, a.grad, a.st, s);
  if (e != cudaSuccess) return e;
  auto k = sigmakin_hs_grad_kernel<P, R>;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, HsGradCfg<P, R>::NT, L::bytes, s>>>(a, cp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_rambo_adjoint(P::NFINAL, a.nevt, a.ecm, a.rnd, a.nrows, a.grad, a.st, s);
}

// mode 0: FP64 helicity-shared adjoint; 1, 2, 5: FP32 helicity-shared adjoint
// (FP64 RAMBO and sums, double-float momentum tables); 3, 4: the per-helicity
// unrolled adjoint in FP64 / FP32 (every helicity recomputes its program)
template <class P>
cudaError_t launch_grad_impl(const GradLaunch& l, int mode, cudaStream_t s) {
  GradArgs a{l.nevt, l.ecm, l.rnd, l.nrows, l.mask, l.gout, l.grad, l.me, l.pp, l.st};
  switch (mode) {
    case 0: return launch_hs_grad_variant<P, double>(a, l.cd, s);
    case 1:
    case 2:
    case 5: return launch_hs_grad_variant<P, float>(a, l.cf, s);
    case 3: return launch_grad_variant<P, double>(a, l.cd, s);
    case 4: return launch_grad_variant<P, float>(a, l.cf, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mg
