// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 1: ee_mumu (e+ e- mu+ mu-)
// 2 Feynman diagrams (2 amplitude terms), 1 colour flows, 6 wavefunctions
// colour-flow coefficients used: [(1+0j)]
#pragma once
namespace mg {
// helicity-shared program: 6 currents in 2 levels, 16 variant slots, 2 amplitudes, 4504 flops per event (all helicities)
static __device__ const HsItem kHsItems1[16] = {{1, 3, -1, 1, 0, 0, {0, 0, 0, 0, 0, 0}, 3, 0, 0}, {1, 3, 1, 1, 0, 1, {0, 0, 0, 0, 0, 0}, 3, 0, 0}, {0, 2, -1, -1, 0, 2, {0, 0, 0, 0, 0, 0}, 2, 0, 0}, {0, 2, 1, -1, 0, 3, {0, 0, 0, 0, 0, 0}, 2, 0, 0}, {1, 0, -1, -1, 0, 4, {0, 0, 0, 0, 0, 0}, 0, 0, 0}, {1, 0, 1, -1, 0, 5, {0, 0, 0, 0, 0, 0}, 0, 0, 0}, {0, 1, -1, 1, 0, 6, {0, 0, 0, 0, 0, 0}, 1, 0, 0}, {0, 1, 1, 1, 0, 7, {0, 0, 0, 0, 0, 0}, 1, 0, 0}, {5, 1, 0, 0, 0, 8, {4, 6, 0, 0, 0, 0}, 0, 0, 0}, {5, 1, 0, 0, 0, 9, {5, 6, 0, 0, 0, 0}, 0, 0, 0}, {5, 1, 0, 0, 0, 10, {4, 7, 0, 0, 0, 0}, 0, 0, 0}, {5, 1, 0, 0, 0, 11, {5, 7, 0, 0, 0, 0}, 0, 0, 0}, {6, 1, 0, 0, 0, 12, {4, 6, 0, 0, 0, 0}, 0, 0, 1}, {6, 1, 0, 0, 0, 13, {5, 6, 0, 0, 0, 0}, 0, 0, 1}, {6, 1, 0, 0, 0, 14, {4, 7, 0, 0, 0, 0}, 0, 0, 1}, {6, 1, 0, 0, 0, 15, {5, 7, 0, 0, 0, 0}, 0, 0, 1}};
static __constant__ HsAmp kHsAmps1[2] = {{1, 0, {0, 1, 4, 0}, {0, 0, 0}}, {2, 0, {0, 1, 5, 0}, {0, 0, 0}}};  // grouped by type
static __device__ const uint16_t kHsSlot1[6][16] = {{0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1}, {2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3}, {4, 4, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5, 5, 5}, {6, 6, 6, 6, 7, 7, 7, 7, 6, 6, 6, 6, 7, 7, 7, 7}, {8, 8, 8, 8, 10, 10, 10, 10, 9, 9, 9, 9, 11, 11, 11, 11}, {12, 12, 12, 12, 14, 14, 14, 14, 13, 13, 13, 13, 15, 15, 15, 15}};
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB1[128] = {0x00003f80, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc1 {
  static constexpr int NPAR = 4;
  static constexpr int NHEL = 16;
  static constexpr int NCOLOR = 1;
  static constexpr int NDIAGRAMS = 2;
  static constexpr int NAMPS = 2;
  // helicity-shared program (tables above)
  static constexpr int HS_NSLOT = 16;
  static constexpr int HS_NITEM = 16;
  static constexpr int HS_NLEVEL = 2;
  static constexpr int HS_NAMP = 2;
  static constexpr int HS_NCUR = 6;
  // operations: current variants per event, amplitudes + flow sums per helicity
  static constexpr long HS_FLOPS_ITEMS = 1240;
  static constexpr long HS_FLOPS_AMP_HEL = 204;
  static __host__ __device__ constexpr int hs_level(int l) {
    constexpr int t[3] = {0, 8, 16};
    return t[l];
  }
  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems1; }
  static __device__ __forceinline__ const HsAmp* hs_amps() { return kHsAmps1; }
  static __device__ __forceinline__ const uint16_t* hs_slots() { return &kHsSlot1[0][0]; }
  static constexpr int HS_NPAT = 1;
  // colour-flow updates of each amplitude pattern: J_s += amp, -amp, i amp, -i amp
  template <class R>
  static __device__ __forceinline__ void hs_flows(int pat, cx<R> amp, cx<R>* J) {
    switch (pat) {
      case 0: J[0] += amp; break;
      default: break;
    }
  }
  // amplitudes of one (event, helicity): operands cur[sl[c * NHEL]], flows into J
  template <class R>
  static __device__ __forceinline__ void hs_amplitudes(const W4<R>* __restrict__ cur, const uint16_t* __restrict__ sl, const R* __restrict__ K, const Couplings<R>& cp, cx<R>* J) {
    W4<R> o0, o1, o2, o3;
    {  // type 1: 1 amplitudes
      int l0 = -1, l1 = -1;
      for (int d = 0; d < 1; ++d) {
        const HsAmp a = kHsAmps1[d];
        if (a.op[0] != l0) { o0 = cur[sl[a.op[0] * NHEL]]; l0 = a.op[0]; }
        if (a.op[1] != l1) { o1 = cur[sl[a.op[1] * NHEL]]; l1 = a.op[1]; }
        o2 = cur[sl[a.op[2] * NHEL]];
        hs_flows<R>(a.pat, FFV1_0<R>(o0, o1, o2, cp.ee), J);
      }
    }
    {  // type 2: 1 amplitudes
      int l0 = -1, l1 = -1;
      for (int d = 1; d < 2; ++d) {
        const HsAmp a = kHsAmps1[d];
        if (a.op[0] != l0) { o0 = cur[sl[a.op[0] * NHEL]]; l0 = a.op[0]; }
        if (a.op[1] != l1) { o1 = cur[sl[a.op[1] * NHEL]]; l1 = a.op[1]; }
        o2 = cur[sl[a.op[2] * NHEL]];
        hs_flows<R>(a.pat, FFV2_4_0<R>(o0, o1, o2, cp.gz, cp.gzl, cp.gzr), J);
      }
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
