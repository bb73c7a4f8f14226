// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 2: gg_tt (g g t t~)
// 3 Feynman diagrams (3 amplitude terms), 2 colour flows, 7 wavefunctions
// colour-flow coefficients used: [-1j, 1j, (1+0j)]
#pragma once
namespace mg {
// helicity-shared program: 7 currents in 2 levels (20 variant slots), 3 amputated currents in 1 chunk(s) of <= 12 slots, 3 amplitudes; 4612 flops per event (all helicities)
static __device__ const HsItem kHsItems2[32] = {{0, {0, 0, 0}, 2, 0, -1, 1, 0, 0, 0, 0}, {1, {0, 0, 0}, 2, 0, 1, 1, 0, 0, 0, 0}, {2, {0, 0, 0}, 2, 1, -1, 1, 0, 1, 0, 0}, {3, {0, 0, 0}, 2, 1, 1, 1, 0, 1, 0, 0}, {4, {0, 0, 0}, 1, 2, -1, 1, 1, 2, 0, 0}, {5, {0, 0, 0}, 1, 2, 1, 1, 1, 2, 0, 0}, {6, {0, 0, 0}, 0, 3, -1, -1, 1, 3, 0, 0}, {7, {0, 0, 0}, 0, 3, 1, -1, 1, 3, 0, 0}, {8, {0, 2, 0}, 7, 0, 0, 0, 0, 4, 5, 0}, {9, {1, 2, 0}, 7, 0, 0, 0, 0, 4, 5, 0}, {10, {0, 3, 0}, 7, 0, 0, 0, 0, 4, 5, 0}, {11, {1, 3, 0}, 7, 0, 0, 0, 0, 4, 5, 0}, {12, {4, 0, 0}, 3, 0, 0, 0, 0, 7, 0, 1}, {13, {4, 1, 0}, 3, 0, 0, 0, 0, 7, 0, 1}, {14, {5, 0, 0}, 3, 0, 0, 0, 0, 7, 0, 1}, {15, {5, 1, 0}, 3, 0, 0, 0, 0, 7, 0, 1}, {16, {4, 2, 0}, 3, 0, 0, 0, 0, 8, 0, 2}, {17, {4, 3, 0}, 3, 0, 0, 0, 0, 8, 0, 2}, {18, {5, 2, 0}, 3, 0, 0, 0, 0, 8, 0, 2}, {19, {5, 3, 0}, 3, 0, 0, 0, 0, 8, 0, 2}, {0, {6, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {1, {6, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {2, {7, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {3, {7, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {4, {6, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {5, {6, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {6, {7, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {7, {7, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {8, {4, 6, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {9, {5, 6, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {10, {4, 7, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {11, {5, 7, 0}, 11, 0, 0, 0, 0, 0, 0, 0}};
static __constant__ int kHsXItem2[2] = {20, 32};  // item ranges of the amputated chunks
static __device__ __align__(16) const uint8_t kHsVar2[256] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 2, 2, 2, 2, 1, 1, 1, 1, 3, 3, 3, 3, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 2, 2, 0, 0, 2, 2, 1, 1, 3, 3, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 4, 4, 2, 2, 6, 6, 1, 1, 5, 5, 3, 3, 7, 7, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 2, 0, 2, 0, 2, 0, 2, 1, 3, 1, 3, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 4, 0, 4, 2, 6, 2, 6, 1, 5, 1, 5, 3, 7, 3, 7, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 4, 2, 6, 0, 4, 2, 6, 1, 5, 3, 7, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15};  // [leg set][helicity]
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB2[128] = {0xc0004180, 0x00000000, 0x00000000, 0x00000000, 0x4180c000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc2 {
  static constexpr int NPAR = 4;
  static constexpr int NHEL = 16;
  static constexpr int NCOLOR = 2;
  static constexpr int NDIAGRAMS = 3;
  static constexpr int NAMPS = 3;
  // helicity-shared program (tables above)
  static constexpr int HS_NSLOT = 20;   // current variant slots per event
  static constexpr int HS_XCAP = 12;    // amputated-current slots per event and chunk
  static constexpr int HS_NXCHUNK = 1;
  static constexpr int HS_XBUFS = 1;   // chunk buffers
  static constexpr int HS_NITEM = 32;
  static constexpr int HS_NLEVEL = 2;
  static constexpr int HS_NAMP = 3;
  static constexpr int HS_NCUR = 7;
  static constexpr int HS_NX = 3;
  // operations: current variants per event, contractions + flow sums per helicity
  static constexpr long HS_FLOPS_ITEMS = 3044;
  static constexpr long HS_FLOPS_AMP_HEL = 98;
  // item ranges of the current levels and of the amputated chunks; amplitude ranges of the chunks
  static __host__ __device__ constexpr int hs_level(int i) {
    constexpr int t[3] = {0, 8, 20};
    return t[i];
  }
  static __device__ __forceinline__ int hs_xitem(int c) { return kHsXItem2[c]; }
  static __device__ __forceinline__ const uint8_t* hs_variants() { return kHsVar2; }
  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems2; }
  // A = sum_i X_i Y_i for the amplitudes of chunk c: X = xb[X slot + variant],
  // Y = cur[Y slot + variant], variant of a leg set S for this helicity = vt[S * NHEL];
  // amplitudes with the same X and colour flows equal up to a phase share one
  // contraction with the phase-weighted sum of their Y;
  // HS_LOCKSTEP(m, n) between amputated currents (amplitudes m and n of the chunk
  // start the previous and the next one)
  template <class R, class CUR, class XB>
  static __device__ __forceinline__ void hs_contract(int c, const CUR& cur, const XB& xb, const uint8_t* __restrict__ vt, cx<R>* J) {
    switch (c) {
      case 0: {
        {
          const W4<R> X = xb[0 + vt[144]];
          dot4_acc<0>(J[1], X, cur[16 + vt[96]]);
        }
        HS_LOCKSTEP(0, 1);
        {
          const W4<R> X = xb[4 + vt[160]];
          dot4_acc<0>(J[0], X, cur[12 + vt[80]]);
        }
        HS_LOCKSTEP(1, 2);
        {
          const W4<R> X = xb[8 + vt[192]];
          { const cx<R> a = dot4(X, cur[8 + vt[48]]); flow_add<3>(J[0], a); flow_add<2>(J[1], a); }
        }
      } break;
      default: break;
    }
  }
  // adjoint of hs_contract: Jb -> atomic adds into curb (operands) and xbb (amputated);
  // full = the warp's lanes are consecutive helicities of its event(s), all good;
  // act = this lane has an (event, helicity) (lanes without one add zeros)
  // PASS bit 0: the operand adjoints Yb (read X); bit 1: the amputated-current
  // adjoints Xb (read Y), so that Xb can overwrite X in a second pass
  template <int PASS, class R, class CUR, class XB>
  static __device__ __forceinline__ void hs_contract_adj(int c, const CUR& cur, const XB& xb, const uint8_t* __restrict__ vt, const cx<R>* Jb, const CUR& curb, const XB& xbb, bool full, int lane, bool act) {
    switch (c) {
      case 0: {
        {
          const int vx = vt[144];
          const W4<R> X = xb[0 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[96];
            W4<R> Y = cur[16 + vy];
            const cx<R> ab = Jb[1];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<9u, false>(Yb, curb, 16 + vy, lane, act);
              } else {
                curb.atomic_add(16 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<6u, false>(Xb, xbb, 0 + vx, lane, act);
            } else {
              xbb.atomic_add(0 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[160];
          const W4<R> X = xb[4 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[80];
            W4<R> Y = cur[12 + vy];
            const cx<R> ab = Jb[0];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<5u, false>(Yb, curb, 12 + vy, lane, act);
              } else {
                curb.atomic_add(12 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<10u, false>(Xb, xbb, 4 + vx, lane, act);
            } else {
              xbb.atomic_add(4 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[192];
          const W4<R> X = xb[8 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[48];
            W4<R> Y = cur[8 + vy];
            const cx<R> ab = mul_i(Jb[0]) + mul_mi(Jb[1]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<3u, false>(Yb, curb, 8 + vy, lane, act);
              } else {
                curb.atomic_add(8 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<12u, false>(Xb, xbb, 8 + vx, lane, act);
            } else {
              xbb.atomic_add(8 + vx, Xb);
            }
          }
        }
      } break;
      default: break;
    }
  }
  static constexpr int NMOM = 9;
  static constexpr int NPROP = 3;
  static constexpr int NFINAL = 2;
  // floating-point operations per helicity: diagram program, CUDA-core colour sum
  static constexpr long FLOPS_AMP = 898;
  static constexpr long FLOPS_CSUM = 25;
  static constexpr double NORM = 1.0 / 256.0;  // 1/(helicity avg x colour avg x symmetry)
  // momentum table: {0 physical / 1 all-outgoing sum, leg mask, mask of legs entering as -p}
  static __host__ __device__ constexpr int mom(int j, int k) {
    constexpr int t[NMOM][3] = {{0, 1, 0}, {0, 2, 0}, {0, 4, 0}, {0, 8, 0}, {1, 1, 1}, {1, 2, 2}, {1, 3, 3}, {1, 5, 1}, {1, 6, 2}};
    return t[j][k];
  }
  // propagators: {momentum entry, 0 gluon / 1 top / 2 photon / 3 Z}
  static __host__ __device__ constexpr int prop(int j, int k) {
    constexpr int t[NPROP][2] = {{6, 0}, {7, 1}, {8, 1}};
    return t[j][k];
  }
  // propagator entries formed from each momentum entry (-1: none)
  static __host__ __device__ constexpr int mom_prop(int j, int k) {
    constexpr int t[NMOM][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {0, -1}, {1, -1}, {2, -1}};
    return t[j][k];
  }
  static __device__ __forceinline__ const uint32_t* colour_bf16_image() { return kColourB2; }
  // colour matrix = CNUM / CDEN (real symmetric)
  static constexpr int CDEN = 3;
  static __host__ __device__ constexpr int cnum(int i, int j) {
    constexpr int t[NCOLOR][NCOLOR] = {{16, -2}, {-2, 16}};
    return t[i][j];
  }
  // Dual amplitudes J_s of one helicity combination (hel[k] = +-1), accumulated
  // through J.add/sub/addi/subi(s, amp) (J_s += amp, -amp, i amp, -i amp);
  // Lock::sync() marks points where a CTA may re-align its warps.
  template <class R, class Acc, class Lock>
  static __device__ __forceinline__ void amplitudes(const R* __restrict__ K, const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, Acc& J) {
    J.zero();
  cx<R> amp;
  const W4<R> w9 = ixxxxx<R>(K + 12, cp.mt, hel[3], -1);
  const W4<R> w0 = vxxxxx<R>(K + 0, hel[0], 1);
  const W4<R> w1 = vxxxxx<R>(K + 4, hel[1], 1);
  const W4<R> w5 = VVV1P0_1<R>(w0, w1, K + 16, K + 20, cp.gs, prop[0]);
  const W4<R> w2 = oxxxxx<R>(K + 8, cp.mt, hel[2], 1);
  amp = FFV1_0<R>(w2, w9, w5, cp.gs);
  J.subi(0, amp);
  J.addi(1, amp);
  const W4<R> w7 = FFV1_2<R>(w2, w0, cp.gs, K + 28, cp.mt, prop[1]);
  amp = FFV1_0<R>(w7, w9, w1, cp.gs);
  Lock::sync();
  J.add(0, amp);
  const W4<R> w3 = FFV1_2<R>(w2, w1, cp.gs, K + 32, cp.mt, prop[2]);
  amp = FFV1_0<R>(w3, w9, w0, cp.gs);
  J.add(1, amp);
  }
  static constexpr bool HAS_GRAD = true;
  // |M_h|^2 of one helicity (colour summed) and its gradient with respect to the
  // physical momenta of the final-state legs, accumulated into pb[4 * leg + mu]
  template <class R>
  static __device__ __forceinline__ R amplitudes_grad(const R* __restrict__ K, const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, R* pb) {
    cx<R> J[NCOLOR];
    #pragma unroll
    for (int s = 0; s < NCOLOR; ++s) J[s] = cx<R>(R(0), R(0));
    cx<R> amp;
    const W4<R> w9 = ixxxxx<R>(K + 12, cp.mt, hel[3], -1);
    const W4<R> w0 = vxxxxx<R>(K + 0, hel[0], 1);
    const W4<R> w1 = vxxxxx<R>(K + 4, hel[1], 1);
    const W4<R> w5 = VVV1P0_1<R>(w0, w1, K + 16, K + 20, cp.gs, prop[0]);
    const W4<R> w2 = oxxxxx<R>(K + 8, cp.mt, hel[2], 1);
    amp = FFV1_0<R>(w2, w9, w5, cp.gs);
    J[0] -= mul_i(amp);
    J[1] += mul_i(amp);
    const W4<R> w7 = FFV1_2<R>(w2, w0, cp.gs, K + 28, cp.mt, prop[1]);
    amp = FFV1_0<R>(w7, w9, w1, cp.gs);
    J[0] += amp;
    const W4<R> w3 = FFV1_2<R>(w2, w1, cp.gs, K + 32, cp.mt, prop[2]);
    amp = FFV1_0<R>(w3, w9, w0, cp.gs);
    J[1] += amp;
    R m2 = R(0);
    cx<R> Jb[NCOLOR];
    { const R tr = R(16) * J[0].re + R(-2) * J[1].re, ti = R(16) * J[0].im + R(-2) * J[1].im; m2 += J[0].re * tr + J[0].im * ti; Jb[0] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    { const R tr = R(-2) * J[0].re + R(16) * J[1].re, ti = R(-2) * J[0].im + R(16) * J[1].im; m2 += J[1].re * tr + J[1].im * ti; Jb[1] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    m2 /= R(CDEN);
    W4<R> w9b = w4_zero<R>();
    W4<R> w0b = w4_zero<R>();
    W4<R> w1b = w4_zero<R>();
    W4<R> w5b = w4_zero<R>();
    W4<R> w2b = w4_zero<R>();
    W4<R> w7b = w4_zero<R>();
    W4<R> w3b = w4_zero<R>();
    cx<R> propb[NPROP];
    #pragma unroll
    for (int j = 0; j < NPROP; ++j) propb[j] = cx<R>(R(0), R(0));
    { const cx<R> ab = Jb[1];
      FFV1_0_adj<R>(w3, w9, w0, cp.gs, ab, w3b, w9b, w0b); }
    { const cx<R> ab = Jb[0];
      FFV1_0_adj<R>(w7, w9, w1, cp.gs, ab, w7b, w9b, w1b); }
    { const cx<R> ab = mul_i(Jb[0]) + mul_mi(Jb[1]);
      FFV1_0_adj<R>(w2, w9, w5, cp.gs, ab, w2b, w9b, w5b); }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w1, cp.gs, K + 32, cp.mt, prop[2], w3b, w2b, w1b, kb, propb[2]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w0, cp.gs, K + 28, cp.mt, prop[1], w7b, w2b, w0b, kb, propb[1]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w0, w1, K + 16, K + 20, cp.gs, prop[0], w5b, w0b, w1b, kb1, kb2, propb[0]);
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[0], false, K + 24, propb[0], kb);
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[1], true, K + 28, propb[1], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[2], true, K + 32, propb[2], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      external_adj<R>(0, K + 12, cp.mt, hel[3], -1, w9b, kb);
    pb[12] += kb[0];
    pb[13] += kb[1];
    pb[14] += kb[2];
    pb[15] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      external_adj<R>(1, K + 8, cp.mt, hel[2], 1, w2b, kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    return m2;
  }
};
}  // namespace mg
