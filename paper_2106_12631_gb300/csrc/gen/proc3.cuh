// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 3: gg_ttg (g g t t~ g)
// 16 Feynman diagrams (18 amplitude terms), 6 colour flows, 26 wavefunctions
// colour-flow coefficients used: [(-1+0j), -1j, 1j, (1+0j)]
#pragma once
namespace mg {
// helicity-shared program: 20 currents in 3 levels, 94 variant slots, 18 amplitudes, 71580 flops per event (all helicities)
static __device__ const HsItem kHsItems3[94] = {{1, 2, -1, 1, 1, 0, {0, 0, 0, 0, 0, 0}, 2, 0, 0}, {1, 2, 1, 1, 1, 1, {0, 0, 0, 0, 0, 0}, 2, 0, 0}, {0, 3, -1, -1, 1, 2, {0, 0, 0, 0, 0, 0}, 3, 0, 0}, {0, 3, 1, -1, 1, 3, {0, 0, 0, 0, 0, 0}, 3, 0, 0}, {2, 0, -1, 1, 0, 4, {0, 0, 0, 0, 0, 0}, 0, 0, 0}, {2, 0, 1, 1, 0, 5, {0, 0, 0, 0, 0, 0}, 0, 0, 0}, {2, 1, -1, 1, 0, 6, {0, 0, 0, 0, 0, 0}, 1, 0, 0}, {2, 1, 1, 1, 0, 7, {0, 0, 0, 0, 0, 0}, 1, 0, 0}, {2, 4, -1, -1, 0, 8, {0, 0, 0, 0, 0, 0}, 4, 0, 0}, {2, 4, 1, -1, 0, 9, {0, 0, 0, 0, 0, 0}, 4, 0, 0}, {7, 0, 0, 0, 0, 10, {6, 8, 0, 0, 0, 0}, 6, 7, 1}, {7, 0, 0, 0, 0, 11, {7, 8, 0, 0, 0, 0}, 6, 7, 1}, {7, 0, 0, 0, 0, 12, {6, 9, 0, 0, 0, 0}, 6, 7, 1}, {7, 0, 0, 0, 0, 13, {7, 9, 0, 0, 0, 0}, 6, 7, 1}, {7, 0, 0, 0, 0, 14, {4, 6, 0, 0, 0, 0}, 9, 6, 6}, {7, 0, 0, 0, 0, 15, {5, 6, 0, 0, 0, 0}, 9, 6, 6}, {7, 0, 0, 0, 0, 16, {4, 7, 0, 0, 0, 0}, 9, 6, 6}, {7, 0, 0, 0, 0, 17, {5, 7, 0, 0, 0, 0}, 9, 6, 6}, {7, 0, 0, 0, 0, 18, {4, 8, 0, 0, 0, 0}, 9, 7, 8}, {7, 0, 0, 0, 0, 19, {5, 8, 0, 0, 0, 0}, 9, 7, 8}, {7, 0, 0, 0, 0, 20, {4, 9, 0, 0, 0, 0}, 9, 7, 8}, {7, 0, 0, 0, 0, 21, {5, 9, 0, 0, 0, 0}, 9, 7, 8}, {8, 0, 0, 0, 0, 22, {6, 4, 8, 4, 6, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 23, {6, 5, 8, 5, 6, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 24, {7, 4, 8, 4, 7, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 25, {7, 5, 8, 5, 7, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 26, {6, 4, 9, 4, 6, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 27, {6, 5, 9, 5, 6, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 28, {7, 4, 9, 4, 7, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 29, {7, 5, 9, 5, 7, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 30, {8, 4, 6, 4, 6, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 31, {8, 5, 6, 5, 6, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 32, {8, 4, 7, 4, 7, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 33, {8, 5, 7, 5, 7, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 34, {9, 4, 6, 4, 6, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 35, {9, 5, 6, 5, 6, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 36, {9, 4, 7, 4, 7, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 37, {9, 5, 7, 5, 7, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 38, {8, 4, 6, 6, 4, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 39, {8, 5, 6, 6, 5, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 40, {8, 4, 7, 7, 4, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 41, {8, 5, 7, 7, 5, 8}, 0, 0, 0}, {8, 0, 0, 0, 0, 42, {9, 4, 6, 6, 4, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 43, {9, 5, 6, 6, 5, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 44, {9, 4, 7, 7, 4, 9}, 0, 0, 0}, {8, 0, 0, 0, 0, 45, {9, 5, 7, 7, 5, 9}, 0, 0, 0}, {3, 0, 0, 0, 0, 46, {0, 4, 0, 0, 0, 0}, 10, 0, 2}, {3, 0, 0, 0, 0, 47, {0, 5, 0, 0, 0, 0}, 10, 0, 2}, {3, 0, 0, 0, 0, 48, {1, 4, 0, 0, 0, 0}, 10, 0, 2}, {3, 0, 0, 0, 0, 49, {1, 5, 0, 0, 0, 0}, 10, 0, 2}, {3, 0, 0, 0, 0, 50, {0, 6, 0, 0, 0, 0}, 17, 0, 9}, {3, 0, 0, 0, 0, 51, {0, 7, 0, 0, 0, 0}, 17, 0, 9}, {3, 0, 0, 0, 0, 52, {1, 6, 0, 0, 0, 0}, 17, 0, 9}, {3, 0, 0, 0, 0, 53, {1, 7, 0, 0, 0, 0}, 17, 0, 9}, {3, 0, 0, 0, 0, 54, {0, 8, 0, 0, 0, 0}, 15, 0, 7}, {3, 0, 0, 0, 0, 55, {1, 8, 0, 0, 0, 0}, 15, 0, 7}, {3, 0, 0, 0, 0, 56, {0, 9, 0, 0, 0, 0}, 15, 0, 7}, {3, 0, 0, 0, 0, 57, {1, 9, 0, 0, 0, 0}, 15, 0, 7}, {4, 0, 0, 0, 0, 58, {2, 8, 0, 0, 0, 0}, 18, 0, 4}, {4, 0, 0, 0, 0, 59, {3, 8, 0, 0, 0, 0}, 18, 0, 4}, {4, 0, 0, 0, 0, 60, {2, 9, 0, 0, 0, 0}, 18, 0, 4}, {4, 0, 0, 0, 0, 61, {3, 9, 0, 0, 0, 0}, 18, 0, 4}, {4, 0, 0, 0, 0, 62, {2, 6, 0, 0, 0, 0}, 19, 0, 5}, {4, 0, 0, 0, 0, 63, {2, 7, 0, 0, 0, 0}, 19, 0, 5}, {4, 0, 0, 0, 0, 64, {3, 6, 0, 0, 0, 0}, 19, 0, 5}, {4, 0, 0, 0, 0, 65, {3, 7, 0, 0, 0, 0}, 19, 0, 5}, {4, 0, 0, 0, 0, 66, {2, 4, 0, 0, 0, 0}, 20, 0, 3}, {4, 0, 0, 0, 0, 67, {2, 5, 0, 0, 0, 0}, 20, 0, 3}, {4, 0, 0, 0, 0, 68, {3, 4, 0, 0, 0, 0}, 20, 0, 3}, {4, 0, 0, 0, 0, 69, {3, 5, 0, 0, 0, 0}, 20, 0, 3}, {7, 0, 0, 0, 0, 70, {4, 10, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 71, {5, 10, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 72, {4, 11, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 73, {5, 11, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 74, {4, 12, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 75, {5, 12, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 76, {4, 13, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 77, {5, 13, 0, 0, 0, 0}, 9, 8, 0}, {7, 0, 0, 0, 0, 78, {14, 8, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 79, {15, 8, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 80, {16, 8, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 81, {17, 8, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 82, {14, 9, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 83, {15, 9, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 84, {16, 9, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 85, {17, 9, 0, 0, 0, 0}, 14, 7, 0}, {7, 0, 0, 0, 0, 86, {18, 6, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 87, {19, 6, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 88, {18, 7, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 89, {19, 7, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 90, {20, 6, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 91, {21, 6, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 92, {20, 7, 0, 0, 0, 0}, 16, 6, 0}, {7, 0, 0, 0, 0, 93, {21, 7, 0, 0, 0, 0}, 16, 6, 0}};
static __constant__ HsAmp kHsAmps3[18] = {{0, 0, {0, 1, 8, 0}, {0, 0, 0}}, {0, 1, {0, 1, 9, 0}, {0, 0, 0}}, {0, 2, {0, 1, 10, 0}, {0, 0, 0}}, {0, 3, {0, 1, 17, 0}, {0, 0, 0}}, {0, 0, {0, 1, 18, 0}, {0, 0, 0}}, {0, 1, {0, 1, 19, 0}, {0, 0, 0}}, {0, 4, {0, 14, 6, 0}, {0, 0, 0}}, {0, 5, {0, 15, 7, 0}, {0, 0, 0}}, {0, 6, {0, 16, 5, 0}, {0, 0, 0}}, {0, 7, {11, 1, 5, 0}, {0, 0, 0}}, {0, 8, {11, 14, 3, 0}, {0, 0, 0}}, {0, 9, {11, 15, 4, 0}, {0, 0, 0}}, {0, 10, {12, 1, 7, 0}, {0, 0, 0}}, {0, 11, {12, 14, 2, 0}, {0, 0, 0}}, {0, 12, {12, 16, 4, 0}, {0, 0, 0}}, {0, 13, {13, 1, 6, 0}, {0, 0, 0}}, {0, 14, {13, 15, 2, 0}, {0, 0, 0}}, {0, 15, {13, 16, 3, 0}, {0, 0, 0}}};  // grouped by type
static __device__ const uint16_t kHsSlot3[20][32] = {{0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1}, {2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3, 2, 2, 3, 3}, {4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5}, {6, 6, 6, 6, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7, 7, 7, 6, 6, 6, 6, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7, 7, 7}, {8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9, 8, 9}, {10, 12, 10, 12, 10, 12, 10, 12, 11, 13, 11, 13, 11, 13, 11, 13, 10, 12, 10, 12, 10, 12, 10, 12, 11, 13, 11, 13, 11, 13, 11, 13}, {14, 14, 14, 14, 14, 14, 14, 14, 16, 16, 16, 16, 16, 16, 16, 16, 15, 15, 15, 15, 15, 15, 15, 15, 17, 17, 17, 17, 17, 17, 17, 17}, {18, 20, 18, 20, 18, 20, 18, 20, 18, 20, 18, 20, 18, 20, 18, 20, 19, 21, 19, 21, 19, 21, 19, 21, 19, 21, 19, 21, 19, 21, 19, 21}, {22, 26, 22, 26, 22, 26, 22, 26, 24, 28, 24, 28, 24, 28, 24, 28, 23, 27, 23, 27, 23, 27, 23, 27, 25, 29, 25, 29, 25, 29, 25, 29}, {30, 34, 30, 34, 30, 34, 30, 34, 32, 36, 32, 36, 32, 36, 32, 36, 31, 35, 31, 35, 31, 35, 31, 35, 33, 37, 33, 37, 33, 37, 33, 37}, {38, 42, 38, 42, 38, 42, 38, 42, 40, 44, 40, 44, 40, 44, 40, 44, 39, 43, 39, 43, 39, 43, 39, 43, 41, 45, 41, 45, 41, 45, 41, 45}, {46, 46, 46, 46, 48, 48, 48, 48, 46, 46, 46, 46, 48, 48, 48, 48, 47, 47, 47, 47, 49, 49, 49, 49, 47, 47, 47, 47, 49, 49, 49, 49}, {50, 50, 50, 50, 52, 52, 52, 52, 51, 51, 51, 51, 53, 53, 53, 53, 50, 50, 50, 50, 52, 52, 52, 52, 51, 51, 51, 51, 53, 53, 53, 53}, {54, 56, 54, 56, 55, 57, 55, 57, 54, 56, 54, 56, 55, 57, 55, 57, 54, 56, 54, 56, 55, 57, 55, 57, 54, 56, 54, 56, 55, 57, 55, 57}, {58, 60, 59, 61, 58, 60, 59, 61, 58, 60, 59, 61, 58, 60, 59, 61, 58, 60, 59, 61, 58, 60, 59, 61, 58, 60, 59, 61, 58, 60, 59, 61}, {62, 62, 64, 64, 62, 62, 64, 64, 63, 63, 65, 65, 63, 63, 65, 65, 62, 62, 64, 64, 62, 62, 64, 64, 63, 63, 65, 65, 63, 63, 65, 65}, {66, 66, 68, 68, 66, 66, 68, 68, 66, 66, 68, 68, 66, 66, 68, 68, 67, 67, 69, 69, 67, 67, 69, 69, 67, 67, 69, 69, 67, 67, 69, 69}, {70, 74, 70, 74, 70, 74, 70, 74, 72, 76, 72, 76, 72, 76, 72, 76, 71, 75, 71, 75, 71, 75, 71, 75, 73, 77, 73, 77, 73, 77, 73, 77}, {78, 82, 78, 82, 78, 82, 78, 82, 80, 84, 80, 84, 80, 84, 80, 84, 79, 83, 79, 83, 79, 83, 79, 83, 81, 85, 81, 85, 81, 85, 81, 85}, {86, 90, 86, 90, 86, 90, 86, 90, 88, 92, 88, 92, 88, 92, 88, 92, 87, 91, 87, 91, 87, 91, 87, 91, 89, 93, 89, 93, 89, 93, 89, 93}};
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB3[128] = {0xc1004280, 0x3f80c100, 0x41203f80, 0x00000000, 0x4280c100, 0x41203f80, 0x3f80c100, 0x00000000, 0x3f80c100, 0xc1004280, 0x3f804120, 0x00000000, 0x41203f80, 0x4280c100, 0xc1003f80, 0x00000000, 0xc1003f80, 0x3f804120, 0xc1004280, 0x00000000, 0x3f804120, 0xc1003f80, 0x4280c100, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc3 {
  static constexpr int NPAR = 5;
  static constexpr int NHEL = 32;
  static constexpr int NCOLOR = 6;
  static constexpr int NDIAGRAMS = 16;
  static constexpr int NAMPS = 18;
  // helicity-shared program (tables above)
  static constexpr int HS_NSLOT = 94;
  static constexpr int HS_NITEM = 94;
  static constexpr int HS_NLEVEL = 3;
  static constexpr int HS_NAMP = 18;
  static constexpr int HS_NCUR = 20;
  // operations: current variants per event, amplitudes + flow sums per helicity
  static constexpr long HS_FLOPS_ITEMS = 13596;
  static constexpr long HS_FLOPS_AMP_HEL = 1812;
  static __host__ __device__ constexpr int hs_level(int l) {
    constexpr int t[4] = {0, 10, 70, 94};
    return t[l];
  }
  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems3; }
  static __device__ __forceinline__ const HsAmp* hs_amps() { return kHsAmps3; }
  static __device__ __forceinline__ const uint16_t* hs_slots() { return &kHsSlot3[0][0]; }
  static constexpr int HS_NPAT = 16;
  // colour-flow updates of each amplitude pattern: J_s += amp, -amp, i amp, -i amp
  template <class R>
  static __device__ __forceinline__ void hs_flows(int pat, cx<R> amp, cx<R>* J) {
    switch (pat) {
      case 0: J[0] -= amp; J[2] += amp; J[4] += amp; J[5] -= amp; break;
      case 1: J[1] -= amp; J[2] += amp; J[3] -= amp; J[4] += amp; break;
      case 2: J[0] += amp; J[1] -= amp; J[3] -= amp; J[5] += amp; break;
      case 3: J[0] -= amp; J[1] += amp; J[3] += amp; J[5] -= amp; break;
      case 4: J[0] -= mul_i(amp); J[2] += mul_i(amp); break;
      case 5: J[1] -= mul_i(amp); J[4] += mul_i(amp); break;
      case 6: J[3] -= mul_i(amp); J[5] += mul_i(amp); break;
      case 7: J[0] -= mul_i(amp); J[1] += mul_i(amp); break;
      case 8: J[0] += amp; break;
      case 9: J[1] += amp; break;
      case 10: J[2] -= mul_i(amp); J[3] += mul_i(amp); break;
      case 11: J[2] += amp; break;
      case 12: J[3] += amp; break;
      case 13: J[4] -= mul_i(amp); J[5] += mul_i(amp); break;
      case 14: J[4] += amp; break;
      case 15: J[5] += amp; break;
      default: break;
    }
  }
  // amplitudes of one (event, helicity): operands cur[sl[c * NHEL]], flows into J
  template <class R>
  static __device__ __forceinline__ void hs_amplitudes(const W4<R>* __restrict__ cur, const uint16_t* __restrict__ sl, const R* __restrict__ K, const Couplings<R>& cp, cx<R>* J) {
    W4<R> o0, o1, o2, o3;
    {  // type 0: 18 amplitudes
      int l0 = -1, l1 = -1;
      for (int d = 0; d < 18; ++d) {
        const HsAmp a = kHsAmps3[d];
        if (a.op[0] != l0) { o0 = cur[sl[a.op[0] * NHEL]]; l0 = a.op[0]; }
        if (a.op[1] != l1) { o1 = cur[sl[a.op[1] * NHEL]]; l1 = a.op[1]; }
        o2 = cur[sl[a.op[2] * NHEL]];
        hs_flows<R>(a.pat, FFV1_0<R>(o0, o1, o2, cp.gs), J);
      }
    }
  }
  static constexpr int NMOM = 21;
  static constexpr int NPROP = 10;
  static constexpr int NFINAL = 3;
  // floating-point operations per helicity: diagram program, CUDA-core colour sum
  static constexpr long FLOPS_AMP = 5220;
  static constexpr long FLOPS_CSUM = 169;
  static constexpr double NORM = 1.0 / 256.0;  // 1/(helicity avg x colour avg x symmetry)
  // momentum table: {0 physical / 1 all-outgoing sum, leg mask, mask of legs entering as -p}
  static __host__ __device__ constexpr int mom(int j, int k) {
    constexpr int t[NMOM][3] = {{0, 1, 0}, {0, 2, 0}, {0, 4, 0}, {0, 8, 0}, {0, 16, 0}, {1, 19, 3}, {1, 2, 2}, {1, 16, 0}, {1, 18, 2}, {1, 1, 1}, {1, 5, 1}, {1, 22, 2}, {1, 7, 3}, {1, 21, 1}, {1, 3, 3}, {1, 20, 0}, {1, 17, 1}, {1, 6, 2}, {1, 7, 4}, {1, 21, 20}, {1, 22, 20}};
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
  static constexpr bool HAS_GRAD = true;
  // |M_h|^2 of one helicity (colour summed) and its gradient with respect to the
  // physical momenta of the final-state legs, accumulated into pb[4 * leg + mu]
  template <class R>
  static __device__ __forceinline__ R amplitudes_grad(const R* __restrict__ K, const cx<R>* __restrict__ prop, const int* hel, const Couplings<R>& cp, R* pb) {
    cx<R> J[NCOLOR];
    #pragma unroll
    for (int s = 0; s < NCOLOR; ++s) J[s] = cx<R>(R(0), R(0));
    cx<R> amp;
    const W4<R> w43 = ixxxxx<R>(K + 12, cp.mt, hel[3], -1);
    const W4<R> w0 = vxxxxx<R>(K + 0, hel[0], 1);
    const W4<R> w1 = vxxxxx<R>(K + 4, hel[1], 1);
    const W4<R> w3 = vxxxxx<R>(K + 16, hel[4], -1);
    const W4<R> w28 = VVVV1P0_1<R>(w0, w1, w3, cp.gs2, prop[0]);
    const W4<R> w2 = oxxxxx<R>(K + 8, cp.mt, hel[2], 1);
    amp = FFV1_0<R>(w2, w43, w28, cp.gs);
    J[0] -= amp;
    J[2] += amp;
    J[4] += amp;
    J[5] -= amp;
    const W4<R> w29 = VVVV3P0_1<R>(w0, w1, w3, cp.gs2, prop[0]);
    amp = FFV1_0<R>(w2, w43, w29, cp.gs);
    J[1] -= amp;
    J[2] += amp;
    J[3] -= amp;
    J[4] += amp;
    const W4<R> w30 = VVVV4P0_1<R>(w0, w1, w3, cp.gs2, prop[0]);
    amp = FFV1_0<R>(w2, w43, w30, cp.gs);
    J[0] += amp;
    J[1] -= amp;
    J[3] -= amp;
    J[5] += amp;
    const W4<R> w8 = VVV1P0_1<R>(w1, w3, K + 24, K + 28, cp.gs, prop[1]);
    const W4<R> w25 = VVV1P0_1<R>(w0, w8, K + 36, K + 32, cp.gs, prop[0]);
    amp = FFV1_0<R>(w2, w43, w25, cp.gs);
    J[0] -= amp;
    J[1] += amp;
    J[3] += amp;
    J[5] -= amp;
    const W4<R> w15 = FFV1_2<R>(w2, w0, cp.gs, K + 40, cp.mt, prop[2]);
    amp = FFV1_0<R>(w15, w43, w8, cp.gs);
    J[0] -= mul_i(amp);
    J[1] += mul_i(amp);
    const W4<R> w9 = FFV1_2<R>(w2, w8, cp.gs, K + 44, cp.mt, prop[3]);
    amp = FFV1_0<R>(w9, w43, w0, cp.gs);
    J[3] -= mul_i(amp);
    J[5] += mul_i(amp);
    const W4<R> w21 = FFV1_2<R>(w15, w1, cp.gs, K + 48, cp.mt, prop[4]);
    amp = FFV1_0<R>(w21, w43, w3, cp.gs);
    J[0] += amp;
    const W4<R> w38 = FFV1_2<R>(w15, w3, cp.gs, K + 52, cp.mt, prop[5]);
    amp = FFV1_0<R>(w38, w43, w1, cp.gs);
    J[1] += amp;
    const W4<R> w13 = VVV1P0_1<R>(w0, w1, K + 36, K + 24, cp.gs, prop[6]);
    const W4<R> w26 = VVV1P0_1<R>(w13, w3, K + 56, K + 28, cp.gs, prop[0]);
    amp = FFV1_0<R>(w2, w43, w26, cp.gs);
    J[0] -= amp;
    J[2] += amp;
    J[4] += amp;
    J[5] -= amp;
    const W4<R> w4 = FFV1_2<R>(w2, w3, cp.gs, K + 60, cp.mt, prop[7]);
    amp = FFV1_0<R>(w4, w43, w13, cp.gs);
    J[4] -= mul_i(amp);
    J[5] += mul_i(amp);
    const W4<R> w20 = FFV1_2<R>(w2, w13, cp.gs, K + 48, cp.mt, prop[4]);
    amp = FFV1_0<R>(w20, w43, w3, cp.gs);
    J[0] -= mul_i(amp);
    J[2] += mul_i(amp);
    const W4<R> w37 = FFV1_2<R>(w4, w0, cp.gs, K + 52, cp.mt, prop[5]);
    amp = FFV1_0<R>(w37, w43, w1, cp.gs);
    J[4] += amp;
    const W4<R> w5 = FFV1_2<R>(w4, w1, cp.gs, K + 44, cp.mt, prop[3]);
    amp = FFV1_0<R>(w5, w43, w0, cp.gs);
    J[5] += amp;
    const W4<R> w17 = VVV1P0_1<R>(w0, w3, K + 36, K + 28, cp.gs, prop[8]);
    const W4<R> w27 = VVV1P0_1<R>(w17, w1, K + 64, K + 24, cp.gs, prop[0]);
    amp = FFV1_0<R>(w2, w43, w27, cp.gs);
    J[1] -= amp;
    J[2] += amp;
    J[3] -= amp;
    J[4] += amp;
    const W4<R> w6 = FFV1_2<R>(w2, w1, cp.gs, K + 68, cp.mt, prop[9]);
    amp = FFV1_0<R>(w6, w43, w17, cp.gs);
    J[2] -= mul_i(amp);
    J[3] += mul_i(amp);
    const W4<R> w39 = FFV1_2<R>(w2, w17, cp.gs, K + 52, cp.mt, prop[5]);
    amp = FFV1_0<R>(w39, w43, w1, cp.gs);
    J[1] -= mul_i(amp);
    J[4] += mul_i(amp);
    const W4<R> w19 = FFV1_2<R>(w6, w0, cp.gs, K + 48, cp.mt, prop[4]);
    amp = FFV1_0<R>(w19, w43, w3, cp.gs);
    J[2] += amp;
    const W4<R> w7 = FFV1_2<R>(w6, w3, cp.gs, K + 44, cp.mt, prop[3]);
    amp = FFV1_0<R>(w7, w43, w0, cp.gs);
    J[3] += amp;
    R m2 = R(0);
    cx<R> Jb[NCOLOR];
    { const R tr = R(64) * J[0].re + R(-8) * J[1].re + R(-8) * J[2].re + R(1) * J[3].re + R(1) * J[4].re + R(10) * J[5].re, ti = R(64) * J[0].im + R(-8) * J[1].im + R(-8) * J[2].im + R(1) * J[3].im + R(1) * J[4].im + R(10) * J[5].im; m2 += J[0].re * tr + J[0].im * ti; Jb[0] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    { const R tr = R(-8) * J[0].re + R(64) * J[1].re + R(1) * J[2].re + R(10) * J[3].re + R(-8) * J[4].re + R(1) * J[5].re, ti = R(-8) * J[0].im + R(64) * J[1].im + R(1) * J[2].im + R(10) * J[3].im + R(-8) * J[4].im + R(1) * J[5].im; m2 += J[1].re * tr + J[1].im * ti; Jb[1] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    { const R tr = R(-8) * J[0].re + R(1) * J[1].re + R(64) * J[2].re + R(-8) * J[3].re + R(10) * J[4].re + R(1) * J[5].re, ti = R(-8) * J[0].im + R(1) * J[1].im + R(64) * J[2].im + R(-8) * J[3].im + R(10) * J[4].im + R(1) * J[5].im; m2 += J[2].re * tr + J[2].im * ti; Jb[2] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    { const R tr = R(1) * J[0].re + R(10) * J[1].re + R(-8) * J[2].re + R(64) * J[3].re + R(1) * J[4].re + R(-8) * J[5].re, ti = R(1) * J[0].im + R(10) * J[1].im + R(-8) * J[2].im + R(64) * J[3].im + R(1) * J[4].im + R(-8) * J[5].im; m2 += J[3].re * tr + J[3].im * ti; Jb[3] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    { const R tr = R(1) * J[0].re + R(-8) * J[1].re + R(10) * J[2].re + R(1) * J[3].re + R(64) * J[4].re + R(-8) * J[5].re, ti = R(1) * J[0].im + R(-8) * J[1].im + R(10) * J[2].im + R(1) * J[3].im + R(64) * J[4].im + R(-8) * J[5].im; m2 += J[4].re * tr + J[4].im * ti; Jb[4] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    { const R tr = R(10) * J[0].re + R(1) * J[1].re + R(1) * J[2].re + R(-8) * J[3].re + R(-8) * J[4].re + R(64) * J[5].re, ti = R(10) * J[0].im + R(1) * J[1].im + R(1) * J[2].im + R(-8) * J[3].im + R(-8) * J[4].im + R(64) * J[5].im; m2 += J[5].re * tr + J[5].im * ti; Jb[5] = cx<R>(R(2) * tr / R(CDEN), R(2) * ti / R(CDEN)); }
    m2 /= R(CDEN);
    W4<R> w43b = w4_zero<R>();
    W4<R> w0b = w4_zero<R>();
    W4<R> w1b = w4_zero<R>();
    W4<R> w3b = w4_zero<R>();
    W4<R> w28b = w4_zero<R>();
    W4<R> w2b = w4_zero<R>();
    W4<R> w29b = w4_zero<R>();
    W4<R> w30b = w4_zero<R>();
    W4<R> w8b = w4_zero<R>();
    W4<R> w25b = w4_zero<R>();
    W4<R> w15b = w4_zero<R>();
    W4<R> w9b = w4_zero<R>();
    W4<R> w21b = w4_zero<R>();
    W4<R> w38b = w4_zero<R>();
    W4<R> w13b = w4_zero<R>();
    W4<R> w26b = w4_zero<R>();
    W4<R> w4b = w4_zero<R>();
    W4<R> w20b = w4_zero<R>();
    W4<R> w37b = w4_zero<R>();
    W4<R> w5b = w4_zero<R>();
    W4<R> w17b = w4_zero<R>();
    W4<R> w27b = w4_zero<R>();
    W4<R> w6b = w4_zero<R>();
    W4<R> w39b = w4_zero<R>();
    W4<R> w19b = w4_zero<R>();
    W4<R> w7b = w4_zero<R>();
    cx<R> propb[NPROP];
    #pragma unroll
    for (int j = 0; j < NPROP; ++j) propb[j] = cx<R>(R(0), R(0));
    { const cx<R> ab = Jb[3];
      FFV1_0_adj<R>(w7, w43, w0, cp.gs, ab, w7b, w43b, w0b); }
    { const cx<R> ab = Jb[2];
      FFV1_0_adj<R>(w19, w43, w3, cp.gs, ab, w19b, w43b, w3b); }
    { const cx<R> ab = mul_i(Jb[1]) + mul_mi(Jb[4]);
      FFV1_0_adj<R>(w39, w43, w1, cp.gs, ab, w39b, w43b, w1b); }
    { const cx<R> ab = mul_i(Jb[2]) + mul_mi(Jb[3]);
      FFV1_0_adj<R>(w6, w43, w17, cp.gs, ab, w6b, w43b, w17b); }
    { const cx<R> ab = -Jb[1] + Jb[2] + -Jb[3] + Jb[4];
      FFV1_0_adj<R>(w2, w43, w27, cp.gs, ab, w2b, w43b, w27b); }
    { const cx<R> ab = Jb[5];
      FFV1_0_adj<R>(w5, w43, w0, cp.gs, ab, w5b, w43b, w0b); }
    { const cx<R> ab = Jb[4];
      FFV1_0_adj<R>(w37, w43, w1, cp.gs, ab, w37b, w43b, w1b); }
    { const cx<R> ab = mul_i(Jb[0]) + mul_mi(Jb[2]);
      FFV1_0_adj<R>(w20, w43, w3, cp.gs, ab, w20b, w43b, w3b); }
    { const cx<R> ab = mul_i(Jb[4]) + mul_mi(Jb[5]);
      FFV1_0_adj<R>(w4, w43, w13, cp.gs, ab, w4b, w43b, w13b); }
    { const cx<R> ab = -Jb[0] + Jb[2] + Jb[4] + -Jb[5];
      FFV1_0_adj<R>(w2, w43, w26, cp.gs, ab, w2b, w43b, w26b); }
    { const cx<R> ab = Jb[1];
      FFV1_0_adj<R>(w38, w43, w1, cp.gs, ab, w38b, w43b, w1b); }
    { const cx<R> ab = Jb[0];
      FFV1_0_adj<R>(w21, w43, w3, cp.gs, ab, w21b, w43b, w3b); }
    { const cx<R> ab = mul_i(Jb[3]) + mul_mi(Jb[5]);
      FFV1_0_adj<R>(w9, w43, w0, cp.gs, ab, w9b, w43b, w0b); }
    { const cx<R> ab = mul_i(Jb[0]) + mul_mi(Jb[1]);
      FFV1_0_adj<R>(w15, w43, w8, cp.gs, ab, w15b, w43b, w8b); }
    { const cx<R> ab = -Jb[0] + Jb[1] + Jb[3] + -Jb[5];
      FFV1_0_adj<R>(w2, w43, w25, cp.gs, ab, w2b, w43b, w25b); }
    { const cx<R> ab = Jb[0] + -Jb[1] + -Jb[3] + Jb[5];
      FFV1_0_adj<R>(w2, w43, w30, cp.gs, ab, w2b, w43b, w30b); }
    { const cx<R> ab = -Jb[1] + Jb[2] + -Jb[3] + Jb[4];
      FFV1_0_adj<R>(w2, w43, w29, cp.gs, ab, w2b, w43b, w29b); }
    { const cx<R> ab = -Jb[0] + Jb[2] + Jb[4] + -Jb[5];
      FFV1_0_adj<R>(w2, w43, w28, cp.gs, ab, w2b, w43b, w28b); }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w6, w3, cp.gs, K + 44, cp.mt, prop[3], w7b, w6b, w3b, kb, propb[3]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w6, w0, cp.gs, K + 48, cp.mt, prop[4], w19b, w6b, w0b, kb, propb[4]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w17, cp.gs, K + 52, cp.mt, prop[5], w39b, w2b, w17b, kb, propb[5]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w1, cp.gs, K + 68, cp.mt, prop[9], w6b, w2b, w1b, kb, propb[9]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w17, w1, K + 64, K + 24, cp.gs, prop[0], w27b, w17b, w1b, kb1, kb2, propb[0]);
    pb[16] += kb1[0];
    pb[17] += kb1[1];
    pb[18] += kb1[2];
    pb[19] += kb1[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w0, w3, K + 36, K + 28, cp.gs, prop[8], w17b, w0b, w3b, kb1, kb2, propb[8]);
    pb[16] += kb2[0];
    pb[17] += kb2[1];
    pb[18] += kb2[2];
    pb[19] += kb2[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w4, w1, cp.gs, K + 44, cp.mt, prop[3], w5b, w4b, w1b, kb, propb[3]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w4, w0, cp.gs, K + 52, cp.mt, prop[5], w37b, w4b, w0b, kb, propb[5]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w13, cp.gs, K + 48, cp.mt, prop[4], w20b, w2b, w13b, kb, propb[4]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w3, cp.gs, K + 60, cp.mt, prop[7], w4b, w2b, w3b, kb, propb[7]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w13, w3, K + 56, K + 28, cp.gs, prop[0], w26b, w13b, w3b, kb1, kb2, propb[0]);
    pb[16] += kb2[0];
    pb[17] += kb2[1];
    pb[18] += kb2[2];
    pb[19] += kb2[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w0, w1, K + 36, K + 24, cp.gs, prop[6], w13b, w0b, w1b, kb1, kb2, propb[6]);
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w15, w3, cp.gs, K + 52, cp.mt, prop[5], w38b, w15b, w3b, kb, propb[5]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w15, w1, cp.gs, K + 48, cp.mt, prop[4], w21b, w15b, w1b, kb, propb[4]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w8, cp.gs, K + 44, cp.mt, prop[3], w9b, w2b, w8b, kb, propb[3]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      FFV1_2_adj<R>(w2, w0, cp.gs, K + 40, cp.mt, prop[2], w15b, w2b, w0b, kb, propb[2]);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w0, w8, K + 36, K + 32, cp.gs, prop[0], w25b, w0b, w8b, kb1, kb2, propb[0]);
    pb[16] += kb2[0];
    pb[17] += kb2[1];
    pb[18] += kb2[2];
    pb[19] += kb2[3];
    }
    { R kb1[4] = {R(0), R(0), R(0), R(0)}, kb2[4] = {R(0), R(0), R(0), R(0)};
      VVV1P0_1_adj<R>(w1, w3, K + 24, K + 28, cp.gs, prop[1], w8b, w1b, w3b, kb1, kb2, propb[1]);
    pb[16] += kb2[0];
    pb[17] += kb2[1];
    pb[18] += kb2[2];
    pb[19] += kb2[3];
    }
    VVVV4P0_1_adj<R>(w0, w1, w3, cp.gs2, prop[0], w30b, w0b, w1b, w3b, propb[0]);
    VVVV3P0_1_adj<R>(w0, w1, w3, cp.gs2, prop[0], w29b, w0b, w1b, w3b, propb[0]);
    VVVV1P0_1_adj<R>(w0, w1, w3, cp.gs2, prop[0], w28b, w0b, w1b, w3b, propb[0]);
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[0], false, K + 20, propb[0], kb);
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[1], false, K + 32, propb[1], kb);
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[2], true, K + 40, propb[2], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[3], true, K + 44, propb[3], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[4], true, K + 48, propb[4], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[5], true, K + 52, propb[5], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[6], false, K + 56, propb[6], kb);
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[7], true, K + 60, propb[7], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[8], false, K + 64, propb[8], kb);
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      prop_adj<R>(prop[9], true, K + 68, propb[9], kb);
    pb[8] += kb[0];
    pb[9] += kb[1];
    pb[10] += kb[2];
    pb[11] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      external_adj<R>(0, K + 12, cp.mt, hel[3], -1, w43b, kb);
    pb[12] += kb[0];
    pb[13] += kb[1];
    pb[14] += kb[2];
    pb[15] += kb[3];
    }
    { R kb[4] = {R(0), R(0), R(0), R(0)};
      external_adj<R>(2, K + 16, R(0), hel[4], -1, w3b, kb);
    pb[16] += kb[0];
    pb[17] += kb[1];
    pb[18] += kb[2];
    pb[19] += kb[3];
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
