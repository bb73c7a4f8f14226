// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 1: ee_mumu (e+ e- mu+ mu-)
// 2 Feynman diagrams (2 amplitude terms), 1 colour flows, 6 wavefunctions
// colour-flow coefficients used: [(1+0j)]
#pragma once
namespace mg {
// helicity-shared program: 6 currents in 2 levels (16 variant slots), 2 amputated currents in 1 chunk(s) of <= 8 slots, 2 amplitudes; 2968 flops per event (all helicities)
static __device__ const HsItem kHsItems1[24] = {{0, {0, 0, 0}, 1, 0, -1, -1, 0, 0, 0, 0}, {1, {0, 0, 0}, 1, 0, 1, -1, 0, 0, 0, 0}, {2, {0, 0, 0}, 0, 1, -1, 1, 0, 1, 0, 0}, {3, {0, 0, 0}, 0, 1, 1, 1, 0, 1, 0, 0}, {4, {0, 0, 0}, 0, 2, -1, -1, 0, 2, 0, 0}, {5, {0, 0, 0}, 0, 2, 1, -1, 0, 2, 0, 0}, {6, {0, 0, 0}, 1, 3, -1, 1, 0, 3, 0, 0}, {7, {0, 0, 0}, 1, 3, 1, 1, 0, 3, 0, 0}, {8, {0, 2, 0}, 5, 1, 0, 0, 0, 0, 0, 0}, {9, {1, 2, 0}, 5, 1, 0, 0, 0, 0, 0, 0}, {10, {0, 3, 0}, 5, 1, 0, 0, 0, 0, 0, 0}, {11, {1, 3, 0}, 5, 1, 0, 0, 0, 0, 0, 0}, {12, {0, 2, 0}, 6, 1, 0, 0, 0, 0, 0, 1}, {13, {1, 2, 0}, 6, 1, 0, 0, 0, 0, 0, 1}, {14, {0, 3, 0}, 6, 1, 0, 0, 0, 0, 0, 1}, {15, {1, 3, 0}, 6, 1, 0, 0, 0, 0, 0, 1}, {0, {6, 4, 0}, 11, 1, 0, 0, 0, 0, 0, 0}, {1, {6, 5, 0}, 11, 1, 0, 0, 0, 0, 0, 0}, {2, {7, 4, 0}, 11, 1, 0, 0, 0, 0, 0, 0}, {3, {7, 5, 0}, 11, 1, 0, 0, 0, 0, 0, 0}, {4, {6, 4, 0}, 12, 0, 0, 0, 0, 0, 0, 0}, {5, {6, 5, 0}, 12, 0, 0, 0, 0, 0, 0, 0}, {6, {7, 4, 0}, 12, 0, 0, 0, 0, 0, 0, 0}, {7, {7, 5, 0}, 12, 0, 0, 0, 0, 0, 0, 0}};
static __constant__ int kHsXItem1[2] = {16, 24};  // item ranges of the amputated chunks
static __device__ __align__(16) const uint8_t kHsVar1[256] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 2, 2, 2, 2, 1, 1, 1, 1, 3, 3, 3, 3, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 2, 2, 0, 0, 2, 2, 1, 1, 3, 3, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 4, 4, 2, 2, 6, 6, 1, 1, 5, 5, 3, 3, 7, 7, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 2, 0, 2, 0, 2, 0, 2, 1, 3, 1, 3, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 4, 0, 4, 2, 6, 2, 6, 1, 5, 1, 5, 3, 7, 3, 7, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 4, 2, 6, 0, 4, 2, 6, 1, 5, 3, 7, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15};  // [leg set][helicity]
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB1[128] = {0x00003f80, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc1 {
  static constexpr int NPAR = 4;
  static constexpr int NHEL = 16;
  static constexpr int NCOLOR = 1;
  static constexpr int NDIAGRAMS = 2;
  static constexpr int NAMPS = 2;
  // helicity-shared program (tables above)
  static constexpr int HS_NSLOT = 16;   // current variant slots per event
  static constexpr int HS_XCAP = 8;    // amputated-current slots per event and chunk
  static constexpr int HS_NXCHUNK = 1;
  static constexpr int HS_XBUFS = 1;   // chunk buffers
  static constexpr int HS_NITEM = 24;
  static constexpr int HS_NLEVEL = 2;
  static constexpr int HS_NAMP = 2;
  static constexpr int HS_NCUR = 6;
  static constexpr int HS_NX = 2;
  // operations: current variants per event, contractions + flow sums per helicity
  static constexpr long HS_FLOPS_ITEMS = 1944;
  static constexpr long HS_FLOPS_AMP_HEL = 64;
  // item ranges of the current levels and of the amputated chunks; amplitude ranges of the chunks
  static __host__ __device__ constexpr int hs_level(int i) {
    constexpr int t[3] = {0, 8, 16};
    return t[i];
  }
  static __device__ __forceinline__ int hs_xitem(int c) { return kHsXItem1[c]; }
  static __device__ __forceinline__ const uint8_t* hs_variants() { return kHsVar1; }
  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems1; }
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
          const W4<R> X = xb[0 + vt[192]];
          dot4_acc<0>(J[0], X, cur[8 + vt[48]]);
        }
        HS_LOCKSTEP(0, 1);
        {
          const W4<R> X = xb[4 + vt[192]];
          dot4_acc<0>(J[0], X, cur[12 + vt[48]]);
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
          const int vx = vt[192];
          const W4<R> X = xb[0 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[48];
            W4<R> Y = cur[8 + vy];
            const cx<R> ab = Jb[0];
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
              w4_warp_reduce_add<12u, false>(Xb, xbb, 0 + vx, lane, act);
            } else {
              xbb.atomic_add(0 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[192];
          const W4<R> X = xb[4 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[48];
            W4<R> Y = cur[12 + vy];
            const cx<R> ab = Jb[0];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<3u, false>(Yb, curb, 12 + vy, lane, act);
              } else {
                curb.atomic_add(12 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<12u, false>(Xb, xbb, 4 + vx, lane, act);
            } else {
              xbb.atomic_add(4 + vx, Xb);
            }
          }
        }
      } break;
      default: break;
    }
  }
  static constexpr int NMOM = 5;
  static constexpr int NPROP = 2;
  static constexpr int NFINAL = 2;
  // floating-point operations per helicity: diagram program, CUDA-core colour sum
  static constexpr long FLOPS_AMP = 604;
  static constexpr long FLOPS_CSUM = 9;
  static constexpr double NORM = 1.0 / 4.0;  // 1/(helicity avg x colour avg x symmetry)
  // momentum table: {0 physical / 1 all-outgoing sum, leg mask, mask of legs entering as -p}
  static __host__ __device__ constexpr int mom(int j, int k) {
    constexpr int t[NMOM][3] = {{0, 1, 0}, {0, 2, 0}, {0, 4, 0}, {0, 8, 0}, {1, 3, 3}};
    return t[j][k];
  }
  // propagators: {momentum entry, 0 gluon / 1 top / 2 photon / 3 Z}
  static __host__ __device__ constexpr int prop(int j, int k) {
    constexpr int t[NPROP][2] = {{4, 2}, {4, 3}};
    return t[j][k];
  }
  // propagator entries formed from each momentum entry (-1: none)
  static __host__ __device__ constexpr int mom_prop(int j, int k) {
    constexpr int t[NMOM][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {0, 1}};
    return t[j][k];
  }
  static __device__ __forceinline__ const uint32_t* colour_bf16_image() { return kColourB1; }
  // colour matrix = CNUM / CDEN (real symmetric)
  static constexpr int CDEN = 1;
  static __host__ __device__ constexpr int cnum(int i, int j) {
    constexpr int t[NCOLOR][NCOLOR] = {{1}};
    return t[i][j];
  }
  // Dual amplitudes J_s of one helicity combination (hel[k] = +-1), accumulated
  // through J.add/sub/addi/subi(s, amp) (J_s += amp, -amp, i amp, -i amp);
  // Lock::sync() marks points where a CTA may re-align its warps.
  template <class R, class Acc, class Lock>
  static __device__ __forceinline__ void amplitudes(const R* __restrict__ K, const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, Acc& J) {
    J.zero();
  cx<R> amp;
  const W4<R> w2 = ixxxxx<R>(K + 8, R(0), hel[2], -1);
  const W4<R> w0 = oxxxxx<R>(K + 0, R(0), hel[0], -1);
  const W4<R> w1 = ixxxxx<R>(K + 4, R(0), hel[1], 1);
  const W4<R> w3 = FFV1P0_3<R>(w0, w1, cp.ee, prop[0]);
  const W4<R> w5 = oxxxxx<R>(K + 12, R(0), hel[3], 1);
  amp = FFV1_0<R>(w5, w2, w3, cp.ee);
  J.add(0, amp);
  const W4<R> w4 = FFV2_4_3<R>(w0, w1, cp.gz, cp.gzl, cp.gzr, prop[1]);
  amp = FFV2_4_0<R>(w5, w2, w4, cp.gz, cp.gzl, cp.gzr);
  Lock::sync();
  J.add(0, amp);
  }
  static constexpr bool HAS_GRAD = false;
};
}  // namespace mg
