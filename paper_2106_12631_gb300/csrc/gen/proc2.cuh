// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 2: gg_tt (g g t t~)
// 3 Feynman diagrams (3 amplitude terms), 2 colour flows, 7 wavefunctions
// colour-flow coefficients used: [-1j, 1j, (1+0j)]
#pragma once
namespace mg {
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB2[128] = {0xc0004180, 0x00000000, 0x00000000, 0x00000000, 0x4180c000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc2 {
  static constexpr int NPAR = 4;
  static constexpr int NHEL = 16;
  static constexpr int NCOLOR = 2;
  static constexpr int NDIAGRAMS = 3;
  static constexpr int NAMPS = 3;
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
};
}  // namespace mg
