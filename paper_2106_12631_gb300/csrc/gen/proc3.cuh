// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 3: gg_ttg (g g t t~ g)
// 16 Feynman diagrams (18 amplitude terms), 6 colour flows, 26 wavefunctions
// colour-flow coefficients used: [(-1+0j), -1j, 1j, (1+0j)]
#pragma once
namespace mg {
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB3[128] = {0xc1004280, 0x3f80c100, 0x41203f80, 0x00000000, 0x4280c100, 0x41203f80, 0x3f80c100, 0x00000000, 0x3f80c100, 0xc1004280, 0x3f804120, 0x00000000, 0x41203f80, 0x4280c100, 0xc1003f80, 0x00000000, 0xc1003f80, 0x3f804120, 0xc1004280, 0x00000000, 0x3f804120, 0xc1003f80, 0x4280c100, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc3 {
  static constexpr int NPAR = 5;
  static constexpr int NHEL = 32;
  static constexpr int NCOLOR = 6;
  static constexpr int NDIAGRAMS = 16;
  static constexpr int NAMPS = 18;
  static constexpr int NMOM = 18;
  static constexpr int NPROP = 10;
  static constexpr int NFINAL = 3;
  // floating-point operations per helicity: diagram program, CUDA-core colour sum
  static constexpr long FLOPS_AMP = 5220;
  static constexpr long FLOPS_CSUM = 169;
  static constexpr double NORM = 1.0 / 256.0;  // 1/(helicity avg x colour avg x symmetry)
  // momentum table: {0 physical / 1 all-outgoing sum, leg mask, mask of legs entering as -p}
  static __host__ __device__ constexpr int mom(int j, int k) {
    constexpr int t[NMOM][3] = {{0, 1, 0}, {0, 2, 0}, {0, 4, 0}, {0, 8, 0}, {0, 16, 0}, {1, 19, 3}, {1, 2, 2}, {1, 16, 0}, {1, 18, 2}, {1, 1, 1}, {1, 5, 1}, {1, 22, 2}, {1, 7, 3}, {1, 21, 1}, {1, 3, 3}, {1, 20, 0}, {1, 17, 1}, {1, 6, 2}};
    return t[j][k];
  }
  // propagators: {momentum entry, 0 gluon / 1 top / 2 photon / 3 Z}
  static __host__ __device__ constexpr int prop(int j, int k) {
    constexpr int t[NPROP][2] = {{5, 0}, {8, 0}, {10, 1}, {11, 1}, {12, 1}, {13, 1}, {14, 0}, {15, 1}, {16, 0}, {17, 1}};
    return t[j][k];
  }
  static __device__ __forceinline__ const uint32_t* colour_bf16_image() { return kColourB3; }
  // colour matrix = CNUM / CDEN (real symmetric)
  static constexpr int CDEN = 9;
  static __host__ __device__ constexpr int cnum(int i, int j) {
    constexpr int t[NCOLOR][NCOLOR] = {{64, -8, -8, 1, 1, 10}, {-8, 64, 1, 10, -8, 1}, {-8, 1, 64, -8, 10, 1}, {1, 10, -8, 64, 1, -8}, {1, -8, 10, 1, 64, -8}, {10, 1, 1, -8, -8, 64}};
    return t[i][j];
  }
  // Dual amplitudes J_s of one helicity combination (hel[k] = +-1), accumulated
  // through J.add/sub/addi/subi(s, amp) (J_s += amp, -amp, i amp, -i amp);
  // Lock::sync() marks points where a CTA may re-align its warps.
  template <class R, class Acc, class Lock>
  static __device__ __forceinline__ void amplitudes(const R* __restrict__ K, const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, Acc& J) {
    J.zero();
  cx<R> amp;
  const W4<R> w43 = ixxxxx<R>(K + 12, cp.mt, hel[3], -1);
  const W4<R> w0 = vxxxxx<R>(K + 0, hel[0], 1);
  const W4<R> w1 = vxxxxx<R>(K + 4, hel[1], 1);
  const W4<R> w3 = vxxxxx<R>(K + 16, hel[4], -1);
  const W4<R> w28 = VVVV1P0_1<R>(w0, w1, w3, cp.gs2, prop[0]);
  const W4<R> w2 = oxxxxx<R>(K + 8, cp.mt, hel[2], 1);
  amp = FFV1_0<R>(w2, w43, w28, cp.gs);
  J.sub(0, amp);
  J.add(2, amp);
  J.add(4, amp);
  J.sub(5, amp);
  const W4<R> w29 = VVVV3P0_1<R>(w0, w1, w3, cp.gs2, prop[0]);
  Lock::sync();
  amp = FFV1_0<R>(w2, w43, w29, cp.gs);
  J.sub(1, amp);
  J.add(2, amp);
  J.sub(3, amp);
  J.add(4, amp);
  const W4<R> w30 = VVVV4P0_1<R>(w0, w1, w3, cp.gs2, prop[0]);
  amp = FFV1_0<R>(w2, w43, w30, cp.gs);
  J.add(0, amp);
  J.sub(1, amp);
  J.sub(3, amp);
  J.add(5, amp);
  const W4<R> w8 = VVV1P0_1<R>(w1, w3, K + 24, K + 28, cp.gs, prop[1]);
  const W4<R> w25 = VVV1P0_1<R>(w0, w8, K + 36, K + 32, cp.gs, prop[0]);
  amp = FFV1_0<R>(w2, w43, w25, cp.gs);
  J.sub(0, amp);
  J.add(1, amp);
  J.add(3, amp);
  J.sub(5, amp);
  const W4<R> w15 = FFV1_2<R>(w2, w0, cp.gs, K + 40, cp.mt, prop[2]);
  amp = FFV1_0<R>(w15, w43, w8, cp.gs);
  Lock::sync();
  J.subi(0, amp);
  J.addi(1, amp);
  const W4<R> w9 = FFV1_2<R>(w2, w8, cp.gs, K + 44, cp.mt, prop[3]);
  amp = FFV1_0<R>(w9, w43, w0, cp.gs);
  J.subi(3, amp);
  J.addi(5, amp);
  const W4<R> w21 = FFV1_2<R>(w15, w1, cp.gs, K + 48, cp.mt, prop[4]);
  amp = FFV1_0<R>(w21, w43, w3, cp.gs);
  J.add(0, amp);
  const W4<R> w38 = FFV1_2<R>(w15, w3, cp.gs, K + 52, cp.mt, prop[5]);
  amp = FFV1_0<R>(w38, w43, w1, cp.gs);
  J.add(1, amp);
  const W4<R> w13 = VVV1P0_1<R>(w0, w1, K + 36, K + 24, cp.gs, prop[6]);
  const W4<R> w26 = VVV1P0_1<R>(w13, w3, K + 56, K + 28, cp.gs, prop[0]);
  Lock::sync();
  amp = FFV1_0<R>(w2, w43, w26, cp.gs);
  J.sub(0, amp);
  J.add(2, amp);
  J.add(4, amp);
  J.sub(5, amp);
  const W4<R> w4 = FFV1_2<R>(w2, w3, cp.gs, K + 60, cp.mt, prop[7]);
  amp = FFV1_0<R>(w4, w43, w13, cp.gs);
  J.subi(4, amp);
  J.addi(5, amp);
  const W4<R> w20 = FFV1_2<R>(w2, w13, cp.gs, K + 48, cp.mt, prop[4]);
  amp = FFV1_0<R>(w20, w43, w3, cp.gs);
  J.subi(0, amp);
  J.addi(2, amp);
  const W4<R> w37 = FFV1_2<R>(w4, w0, cp.gs, K + 52, cp.mt, prop[5]);
  amp = FFV1_0<R>(w37, w43, w1, cp.gs);
  J.add(4, amp);
  const W4<R> w5 = FFV1_2<R>(w4, w1, cp.gs, K + 44, cp.mt, prop[3]);
  Lock::sync();
  amp = FFV1_0<R>(w5, w43, w0, cp.gs);
  J.add(5, amp);
  const W4<R> w17 = VVV1P0_1<R>(w0, w3, K + 36, K + 28, cp.gs, prop[8]);
  const W4<R> w27 = VVV1P0_1<R>(w17, w1, K + 64, K + 24, cp.gs, prop[0]);
  amp = FFV1_0<R>(w2, w43, w27, cp.gs);
  J.sub(1, amp);
  J.add(2, amp);
  J.sub(3, amp);
  J.add(4, amp);
  const W4<R> w6 = FFV1_2<R>(w2, w1, cp.gs, K + 68, cp.mt, prop[9]);
  amp = FFV1_0<R>(w6, w43, w17, cp.gs);
  J.subi(2, amp);
  J.addi(3, amp);
  const W4<R> w39 = FFV1_2<R>(w2, w17, cp.gs, K + 52, cp.mt, prop[5]);
  amp = FFV1_0<R>(w39, w43, w1, cp.gs);
  Lock::sync();
  J.subi(1, amp);
  J.addi(4, amp);
  const W4<R> w19 = FFV1_2<R>(w6, w0, cp.gs, K + 48, cp.mt, prop[4]);
  amp = FFV1_0<R>(w19, w43, w3, cp.gs);
  J.add(2, amp);
  const W4<R> w7 = FFV1_2<R>(w6, w3, cp.gs, K + 44, cp.mt, prop[3]);
  amp = FFV1_0<R>(w7, w43, w0, cp.gs);
  J.add(3, amp);
  }
};
}  // namespace mg
