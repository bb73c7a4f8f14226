// GENERATED by paper_2106_12631_gb300/gen/procgen.py -- do not edit.
// Process 3: gg_ttg (g g t t~ g)
// 16 Feynman diagrams (18 amplitude terms), 6 colour flows, 26 wavefunctions
// colour-flow coefficients used: [(-1+0j), -1j, 1j, (1+0j)]
#pragma once
namespace mg {
// helicity-shared program: 20 currents in 3 levels (94 variant slots), 13 amputated currents in 1 chunk(s) of <= 100 slots, 18 amplitudes; 37916 flops per event (all helicities)
static __device__ const HsItem kHsItems3[194] = {{0, {0, 0, 0}, 2, 0, -1, 1, 0, 0, 0, 0}, {1, {0, 0, 0}, 2, 0, 1, 1, 0, 0, 0, 0}, {2, {0, 0, 0}, 2, 1, -1, 1, 0, 1, 0, 0}, {3, {0, 0, 0}, 2, 1, 1, 1, 0, 1, 0, 0}, {4, {0, 0, 0}, 1, 2, -1, 1, 1, 2, 0, 0}, {5, {0, 0, 0}, 1, 2, 1, 1, 1, 2, 0, 0}, {6, {0, 0, 0}, 0, 3, -1, -1, 1, 3, 0, 0}, {7, {0, 0, 0}, 0, 3, 1, -1, 1, 3, 0, 0}, {8, {0, 0, 0}, 2, 4, -1, -1, 0, 4, 0, 0}, {9, {0, 0, 0}, 2, 4, 1, -1, 0, 4, 0, 0}, {10, {6, 0, 0}, 4, 0, 0, 0, 0, 18, 0, 3}, {11, {6, 1, 0}, 4, 0, 0, 0, 0, 18, 0, 3}, {12, {7, 0, 0}, 4, 0, 0, 0, 0, 18, 0, 3}, {13, {7, 1, 0}, 4, 0, 0, 0, 0, 18, 0, 3}, {14, {6, 2, 0}, 4, 0, 0, 0, 0, 19, 0, 5}, {15, {6, 3, 0}, 4, 0, 0, 0, 0, 19, 0, 5}, {16, {7, 2, 0}, 4, 0, 0, 0, 0, 19, 0, 5}, {17, {7, 3, 0}, 4, 0, 0, 0, 0, 19, 0, 5}, {18, {6, 8, 0}, 4, 0, 0, 0, 0, 20, 0, 4}, {19, {7, 8, 0}, 4, 0, 0, 0, 0, 20, 0, 4}, {20, {6, 9, 0}, 4, 0, 0, 0, 0, 20, 0, 4}, {21, {7, 9, 0}, 4, 0, 0, 0, 0, 20, 0, 4}, {22, {0, 2, 0}, 7, 0, 0, 0, 0, 9, 6, 6}, {23, {1, 2, 0}, 7, 0, 0, 0, 0, 9, 6, 6}, {24, {0, 3, 0}, 7, 0, 0, 0, 0, 9, 6, 6}, {25, {1, 3, 0}, 7, 0, 0, 0, 0, 9, 6, 6}, {26, {0, 8, 0}, 7, 0, 0, 0, 0, 9, 7, 8}, {27, {1, 8, 0}, 7, 0, 0, 0, 0, 9, 7, 8}, {28, {0, 9, 0}, 7, 0, 0, 0, 0, 9, 7, 8}, {29, {1, 9, 0}, 7, 0, 0, 0, 0, 9, 7, 8}, {30, {2, 8, 0}, 7, 0, 0, 0, 0, 6, 7, 1}, {31, {3, 8, 0}, 7, 0, 0, 0, 0, 6, 7, 1}, {32, {2, 9, 0}, 7, 0, 0, 0, 0, 6, 7, 1}, {33, {3, 9, 0}, 7, 0, 0, 0, 0, 6, 7, 1}, {34, {2, 0, 8}, 8, 0, 0, 0, 0, 0, 0, 0}, {35, {2, 1, 8}, 8, 0, 0, 0, 0, 0, 0, 0}, {36, {3, 0, 8}, 8, 0, 0, 0, 0, 0, 0, 0}, {37, {3, 1, 8}, 8, 0, 0, 0, 0, 0, 0, 0}, {38, {2, 0, 9}, 8, 0, 0, 0, 0, 0, 0, 0}, {39, {2, 1, 9}, 8, 0, 0, 0, 0, 0, 0, 0}, {40, {3, 0, 9}, 8, 0, 0, 0, 0, 0, 0, 0}, {41, {3, 1, 9}, 8, 0, 0, 0, 0, 0, 0, 0}, {42, {8, 0, 2}, 8, 0, 0, 0, 0, 0, 0, 0}, {43, {8, 1, 2}, 8, 0, 0, 0, 0, 0, 0, 0}, {44, {8, 0, 3}, 8, 0, 0, 0, 0, 0, 0, 0}, {45, {8, 1, 3}, 8, 0, 0, 0, 0, 0, 0, 0}, {46, {9, 0, 2}, 8, 0, 0, 0, 0, 0, 0, 0}, {47, {9, 1, 2}, 8, 0, 0, 0, 0, 0, 0, 0}, {48, {9, 0, 3}, 8, 0, 0, 0, 0, 0, 0, 0}, {49, {9, 1, 3}, 8, 0, 0, 0, 0, 0, 0, 0}, {50, {8, 2, 0}, 8, 0, 0, 0, 0, 0, 0, 0}, {51, {8, 2, 1}, 8, 0, 0, 0, 0, 0, 0, 0}, {52, {8, 3, 0}, 8, 0, 0, 0, 0, 0, 0, 0}, {53, {8, 3, 1}, 8, 0, 0, 0, 0, 0, 0, 0}, {54, {9, 2, 0}, 8, 0, 0, 0, 0, 0, 0, 0}, {55, {9, 2, 1}, 8, 0, 0, 0, 0, 0, 0, 0}, {56, {9, 3, 0}, 8, 0, 0, 0, 0, 0, 0, 0}, {57, {9, 3, 1}, 8, 0, 0, 0, 0, 0, 0, 0}, {58, {4, 0, 0}, 3, 0, 0, 0, 0, 10, 0, 2}, {59, {4, 1, 0}, 3, 0, 0, 0, 0, 10, 0, 2}, {60, {5, 0, 0}, 3, 0, 0, 0, 0, 10, 0, 2}, {61, {5, 1, 0}, 3, 0, 0, 0, 0, 10, 0, 2}, {62, {4, 2, 0}, 3, 0, 0, 0, 0, 17, 0, 9}, {63, {4, 3, 0}, 3, 0, 0, 0, 0, 17, 0, 9}, {64, {5, 2, 0}, 3, 0, 0, 0, 0, 17, 0, 9}, {65, {5, 3, 0}, 3, 0, 0, 0, 0, 17, 0, 9}, {66, {4, 8, 0}, 3, 0, 0, 0, 0, 15, 0, 7}, {67, {5, 8, 0}, 3, 0, 0, 0, 0, 15, 0, 7}, {68, {4, 9, 0}, 3, 0, 0, 0, 0, 15, 0, 7}, {69, {5, 9, 0}, 3, 0, 0, 0, 0, 15, 0, 7}, {70, {0, 30, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {71, {1, 30, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {72, {0, 31, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {73, {1, 31, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {74, {0, 32, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {75, {1, 32, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {76, {0, 33, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {77, {1, 33, 0}, 7, 0, 0, 0, 0, 9, 8, 0}, {78, {22, 8, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {79, {23, 8, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {80, {24, 8, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {81, {25, 8, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {82, {22, 9, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {83, {23, 9, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {84, {24, 9, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {85, {25, 9, 0}, 7, 0, 0, 0, 0, 14, 7, 0}, {86, {26, 2, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {87, {27, 2, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {88, {26, 3, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {89, {27, 3, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {90, {28, 2, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {91, {29, 2, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {92, {28, 3, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {93, {29, 3, 0}, 7, 0, 0, 0, 0, 16, 6, 0}, {0, {14, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {1, {14, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {2, {15, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {3, {15, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {4, {16, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {5, {16, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {6, {17, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {7, {17, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {8, {10, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {9, {11, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {10, {10, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {11, {11, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {12, {12, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {13, {13, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {14, {12, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {15, {13, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {16, {6, 22, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {17, {6, 23, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {18, {6, 24, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {19, {6, 25, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {20, {7, 22, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {21, {7, 23, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {22, {7, 24, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {23, {7, 25, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {24, {18, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {25, {18, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {26, {19, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {27, {19, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {28, {20, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {29, {20, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {30, {21, 0, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {31, {21, 1, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {32, {6, 26, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {33, {6, 27, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {34, {7, 26, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {35, {7, 27, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {36, {6, 28, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {37, {6, 29, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {38, {7, 28, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {39, {7, 29, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {40, {10, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {41, {11, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {42, {12, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {43, {13, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {44, {10, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {45, {11, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {46, {12, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {47, {13, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {48, {18, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {49, {18, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {50, {19, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {51, {19, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {52, {20, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {53, {20, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {54, {21, 2, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {55, {21, 3, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {56, {14, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {57, {15, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {58, {16, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {59, {17, 8, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {60, {14, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {61, {15, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {62, {16, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {63, {17, 9, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {64, {6, 30, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {65, {6, 31, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {66, {7, 30, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {67, {7, 31, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {68, {6, 32, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {69, {6, 33, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {70, {7, 32, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {71, {7, 33, 0}, 10, 0, 0, 0, 0, 0, 0, 0}, {72, {4, 6, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {73, {5, 6, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {74, {4, 7, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {75, {5, 7, 0}, 11, 0, 0, 0, 0, 0, 0, 0}, {76, {4, 22, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {77, {4, 23, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {78, {4, 24, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {79, {4, 25, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {80, {5, 22, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {81, {5, 23, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {82, {5, 24, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {83, {5, 25, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {84, {4, 26, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {85, {4, 27, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {86, {5, 26, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {87, {5, 27, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {88, {4, 28, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {89, {4, 29, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {90, {5, 28, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {91, {5, 29, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {92, {4, 30, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {93, {4, 31, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {94, {5, 30, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {95, {5, 31, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {96, {4, 32, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {97, {4, 33, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {98, {5, 32, 0}, 9, 0, 0, 0, 0, 0, 0, 0}, {99, {5, 33, 0}, 9, 0, 0, 0, 0, 0, 0, 0}};
static __constant__ int kHsXItem3[2] = {94, 194};  // item ranges of the amputated chunks
static __device__ __align__(16) const uint8_t kHsVar3[1024] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 2, 2, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 3, 3, 3, 3, 3, 3, 3, 3, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 2, 2, 2, 2, 0, 0, 0, 0, 2, 2, 2, 2, 1, 1, 1, 1, 3, 3, 3, 3, 1, 1, 1, 1, 3, 3, 3, 3, 0, 0, 0, 0, 2, 2, 2, 2, 1, 1, 1, 1, 3, 3, 3, 3, 0, 0, 0, 0, 2, 2, 2, 2, 1, 1, 1, 1, 3, 3, 3, 3, 0, 0, 0, 0, 4, 4, 4, 4, 2, 2, 2, 2, 6, 6, 6, 6, 1, 1, 1, 1, 5, 5, 5, 5, 3, 3, 3, 3, 7, 7, 7, 7, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 2, 2, 0, 0, 2, 2, 0, 0, 2, 2, 0, 0, 2, 2, 1, 1, 3, 3, 1, 1, 3, 3, 1, 1, 3, 3, 1, 1, 3, 3, 0, 0, 2, 2, 0, 0, 2, 2, 1, 1, 3, 3, 1, 1, 3, 3, 0, 0, 2, 2, 0, 0, 2, 2, 1, 1, 3, 3, 1, 1, 3, 3, 0, 0, 4, 4, 0, 0, 4, 4, 2, 2, 6, 6, 2, 2, 6, 6, 1, 1, 5, 5, 1, 1, 5, 5, 3, 3, 7, 7, 3, 3, 7, 7, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 2, 2, 1, 1, 3, 3, 0, 0, 4, 4, 2, 2, 6, 6, 0, 0, 4, 4, 2, 2, 6, 6, 1, 1, 5, 5, 3, 3, 7, 7, 1, 1, 5, 5, 3, 3, 7, 7, 0, 0, 4, 4, 2, 2, 6, 6, 1, 1, 5, 5, 3, 3, 7, 7, 0, 0, 4, 4, 2, 2, 6, 6, 1, 1, 5, 5, 3, 3, 7, 7, 0, 0, 8, 8, 4, 4, 12, 12, 2, 2, 10, 10, 6, 6, 14, 14, 1, 1, 9, 9, 5, 5, 13, 13, 3, 3, 11, 11, 7, 7, 15, 15, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 2, 0, 2, 0, 2, 0, 2, 0, 2, 0, 2, 0, 2, 0, 2, 1, 3, 1, 3, 1, 3, 1, 3, 1, 3, 1, 3, 1, 3, 1, 3, 0, 2, 0, 2, 0, 2, 0, 2, 1, 3, 1, 3, 1, 3, 1, 3, 0, 2, 0, 2, 0, 2, 0, 2, 1, 3, 1, 3, 1, 3, 1, 3, 0, 4, 0, 4, 0, 4, 0, 4, 2, 6, 2, 6, 2, 6, 2, 6, 1, 5, 1, 5, 1, 5, 1, 5, 3, 7, 3, 7, 3, 7, 3, 7, 0, 2, 0, 2, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 2, 0, 2, 1, 3, 1, 3, 0, 4, 0, 4, 2, 6, 2, 6, 0, 4, 0, 4, 2, 6, 2, 6, 1, 5, 1, 5, 3, 7, 3, 7, 1, 5, 1, 5, 3, 7, 3, 7, 0, 4, 0, 4, 2, 6, 2, 6, 1, 5, 1, 5, 3, 7, 3, 7, 0, 4, 0, 4, 2, 6, 2, 6, 1, 5, 1, 5, 3, 7, 3, 7, 0, 8, 0, 8, 4, 12, 4, 12, 2, 10, 2, 10, 6, 14, 6, 14, 1, 9, 1, 9, 5, 13, 5, 13, 3, 11, 3, 11, 7, 15, 7, 15, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 2, 1, 3, 0, 4, 2, 6, 0, 4, 2, 6, 0, 4, 2, 6, 0, 4, 2, 6, 1, 5, 3, 7, 1, 5, 3, 7, 1, 5, 3, 7, 1, 5, 3, 7, 0, 4, 2, 6, 0, 4, 2, 6, 1, 5, 3, 7, 1, 5, 3, 7, 0, 4, 2, 6, 0, 4, 2, 6, 1, 5, 3, 7, 1, 5, 3, 7, 0, 8, 4, 12, 0, 8, 4, 12, 2, 10, 6, 14, 2, 10, 6, 14, 1, 9, 5, 13, 1, 9, 5, 13, 3, 11, 7, 15, 3, 11, 7, 15, 0, 4, 2, 6, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 4, 2, 6, 1, 5, 3, 7, 0, 8, 4, 12, 2, 10, 6, 14, 0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15, 1, 9, 5, 13, 3, 11, 7, 15, 0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15, 0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15, 0, 16, 8, 24, 4, 20, 12, 28, 2, 18, 10, 26, 6, 22, 14, 30, 1, 17, 9, 25, 5, 21, 13, 29, 3, 19, 11, 27, 7, 23, 15, 31};  // [leg set][helicity]
// colour-matrix numerators as the BF16 B operand of the tensor-core colour sum
static __device__ __align__(16) const uint32_t kColourB3[128] = {0xc1004280, 0x3f80c100, 0x41203f80, 0x00000000, 0x4280c100, 0x41203f80, 0x3f80c100, 0x00000000, 0x3f80c100, 0xc1004280, 0x3f804120, 0x00000000, 0x41203f80, 0x4280c100, 0xc1003f80, 0x00000000, 0xc1003f80, 0x3f804120, 0xc1004280, 0x00000000, 0x3f804120, 0xc1003f80, 0x4280c100, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000, 0x00000000};
struct Proc3 {
  static constexpr int NPAR = 5;
  static constexpr int NHEL = 32;
  static constexpr int NCOLOR = 6;
  static constexpr int NDIAGRAMS = 16;
  static constexpr int NAMPS = 18;
  // helicity-shared program (tables above)
  static constexpr int HS_NSLOT = 94;   // current variant slots per event
  static constexpr int HS_XCAP = 100;    // amputated-current slots per event and chunk
  static constexpr int HS_NXCHUNK = 1;
  static constexpr int HS_XBUFS = 1;   // chunk buffers
  static constexpr int HS_NITEM = 194;
  static constexpr int HS_NLEVEL = 3;
  static constexpr int HS_NAMP = 18;
  static constexpr int HS_NCUR = 20;
  static constexpr int HS_NX = 13;
  // operations: current variants per event, contractions + flow sums per helicity
  static constexpr long HS_FLOPS_ITEMS = 20828;
  static constexpr long HS_FLOPS_AMP_HEL = 534;
  // item ranges of the current levels and of the amputated chunks; amplitude ranges of the chunks
  static __host__ __device__ constexpr int hs_level(int i) {
    constexpr int t[4] = {0, 10, 70, 94};
    return t[i];
  }
  static __device__ __forceinline__ int hs_xitem(int c) { return kHsXItem3[c]; }
  static __device__ __forceinline__ const uint8_t* hs_variants() { return kHsVar3; }
  static __device__ __forceinline__ const HsItem* hs_items() { return kHsItems3; }
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
          const W4<R> X = xb[0 + vt[352]];
          dot4_acc<0>(J[4], X, cur[66 + vt[640]]);
        }
        HS_LOCKSTEP(0, 1);
        {
          const W4<R> X = xb[8 + vt[352]];
          dot4_acc<0>(J[5], X, cur[66 + vt[640]]);
        }
        HS_LOCKSTEP(1, 2);
        {
          const W4<R> X = xb[16 + vt[352]];
          { const cx<R> a = dot4(X, cur[66 + vt[640]]); flow_add<3>(J[4], a); flow_add<2>(J[5], a); }
        }
        HS_LOCKSTEP(2, 3);
        {
          const W4<R> X = xb[24 + vt[800]];
          dot4_acc<0>(J[2], X, cur[62 + vt[192]]);
        }
        HS_LOCKSTEP(3, 4);
        {
          const W4<R> X = xb[32 + vt[800]];
          { const cx<R> a = dot4(X, cur[62 + vt[192]]); flow_add<3>(J[2], a); flow_add<2>(J[3], a); }
        }
        HS_LOCKSTEP(4, 5);
        {
          const W4<R> X = xb[40 + vt[800]];
          dot4_acc<0>(J[3], X, cur[62 + vt[192]]);
        }
        HS_LOCKSTEP(5, 6);
        {
          const W4<R> X = xb[48 + vt[832]];
          dot4_acc<0>(J[0], X, cur[58 + vt[160]]);
        }
        HS_LOCKSTEP(6, 7);
        {
          const W4<R> X = xb[56 + vt[832]];
          dot4_acc<0>(J[1], X, cur[58 + vt[160]]);
        }
        HS_LOCKSTEP(7, 8);
        {
          const W4<R> X = xb[64 + vt[832]];
          { const cx<R> a = dot4(X, cur[58 + vt[160]]); flow_add<3>(J[0], a); flow_add<2>(J[1], a); }
        }
        HS_LOCKSTEP(8, 9);
        {
          const W4<R> X = xb[72 + vt[384]];
          {
            W4<R> Y = cur[34 + vt[608]];
            Y = w4_add(Y, cur[78 + vt[608]]);
            const cx<R> a = dot4(X, Y); flow_add<1>(J[0], a); flow_add<0>(J[2], a); flow_add<0>(J[4], a); flow_add<1>(J[5], a);
          }
          {
            W4<R> Y = cur[42 + vt[608]];
            Y = w4_add(Y, cur[86 + vt[608]]);
            const cx<R> a = dot4(X, Y); flow_add<1>(J[1], a); flow_add<0>(J[2], a); flow_add<1>(J[3], a); flow_add<0>(J[4], a);
          }
          {
            W4<R> Y = cur[50 + vt[608]];
            Y = w4_sub(Y, cur[70 + vt[608]]);
            const cx<R> a = dot4(X, Y); flow_add<0>(J[0], a); flow_add<1>(J[1], a); flow_add<1>(J[3], a); flow_add<0>(J[5], a);
          }
        }
        HS_LOCKSTEP(9, 15);
        {
          const W4<R> X = xb[76 + vt[224]];
          { const cx<R> a = dot4(X, cur[18 + vt[768]]); flow_add<3>(J[0], a); flow_add<2>(J[2], a); }
        }
        HS_LOCKSTEP(15, 16);
        {
          const W4<R> X = xb[84 + vt[672]];
          { const cx<R> a = dot4(X, cur[14 + vt[320]]); flow_add<3>(J[1], a); flow_add<2>(J[4], a); }
        }
        HS_LOCKSTEP(16, 17);
        {
          const W4<R> X = xb[92 + vt[704]];
          { const cx<R> a = dot4(X, cur[10 + vt[288]]); flow_add<3>(J[3], a); flow_add<2>(J[5], a); }
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
          const int vx = vt[352];
          const W4<R> X = xb[0 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[640];
            W4<R> Y = cur[66 + vy];
            const cx<R> ab = Jb[4];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<26u, false>(Yb, curb, 66 + vy, lane, act);
              } else {
                curb.atomic_add(66 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<5u, false>(Xb, xbb, 0 + vx, lane, act);
            } else {
              xbb.atomic_add(0 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[352];
          const W4<R> X = xb[8 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[640];
            W4<R> Y = cur[66 + vy];
            const cx<R> ab = Jb[5];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<26u, false>(Yb, curb, 66 + vy, lane, act);
              } else {
                curb.atomic_add(66 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<5u, false>(Xb, xbb, 8 + vx, lane, act);
            } else {
              xbb.atomic_add(8 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[352];
          const W4<R> X = xb[16 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[640];
            W4<R> Y = cur[66 + vy];
            const cx<R> ab = mul_i(Jb[4]) + mul_mi(Jb[5]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<26u, false>(Yb, curb, 66 + vy, lane, act);
              } else {
                curb.atomic_add(66 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<5u, false>(Xb, xbb, 16 + vx, lane, act);
            } else {
              xbb.atomic_add(16 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[800];
          const W4<R> X = xb[24 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[192];
            W4<R> Y = cur[62 + vy];
            const cx<R> ab = Jb[2];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<19u, false>(Yb, curb, 62 + vy, lane, act);
              } else {
                curb.atomic_add(62 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<12u, false>(Xb, xbb, 24 + vx, lane, act);
            } else {
              xbb.atomic_add(24 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[800];
          const W4<R> X = xb[32 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[192];
            W4<R> Y = cur[62 + vy];
            const cx<R> ab = mul_i(Jb[2]) + mul_mi(Jb[3]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<19u, false>(Yb, curb, 62 + vy, lane, act);
              } else {
                curb.atomic_add(62 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<12u, false>(Xb, xbb, 32 + vx, lane, act);
            } else {
              xbb.atomic_add(32 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[800];
          const W4<R> X = xb[40 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[192];
            W4<R> Y = cur[62 + vy];
            const cx<R> ab = Jb[3];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<19u, false>(Yb, curb, 62 + vy, lane, act);
              } else {
                curb.atomic_add(62 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<12u, false>(Xb, xbb, 40 + vx, lane, act);
            } else {
              xbb.atomic_add(40 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[832];
          const W4<R> X = xb[48 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[160];
            W4<R> Y = cur[58 + vy];
            const cx<R> ab = Jb[0];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<11u, false>(Yb, curb, 58 + vy, lane, act);
              } else {
                curb.atomic_add(58 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<20u, false>(Xb, xbb, 48 + vx, lane, act);
            } else {
              xbb.atomic_add(48 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[832];
          const W4<R> X = xb[56 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[160];
            W4<R> Y = cur[58 + vy];
            const cx<R> ab = Jb[1];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<11u, false>(Yb, curb, 58 + vy, lane, act);
              } else {
                curb.atomic_add(58 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<20u, false>(Xb, xbb, 56 + vx, lane, act);
            } else {
              xbb.atomic_add(56 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[832];
          const W4<R> X = xb[64 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[160];
            W4<R> Y = cur[58 + vy];
            const cx<R> ab = mul_i(Jb[0]) + mul_mi(Jb[1]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<11u, false>(Yb, curb, 58 + vy, lane, act);
              } else {
                curb.atomic_add(58 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<20u, false>(Xb, xbb, 64 + vx, lane, act);
            } else {
              xbb.atomic_add(64 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[384];
          const W4<R> X = xb[72 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[608];
            W4<R> Y = cur[34 + vy];
            Y = w4_add(Y, cur[78 + vy]);
            const cx<R> ab = -Jb[0] + Jb[2] + Jb[4] + -Jb[5];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<6u, false>(Yb, curb, 34 + vy, lane, act);
              } else {
                curb.atomic_add(34 + vy, Yb);
              }
              if (full) {
                w4_warp_reduce_add<6u, false>(Yb, curb, 78 + vy, lane, act);
              } else {
                curb.atomic_add(78 + vy, Yb);
              }
            }
          }
          {
            const int vy = vt[608];
            W4<R> Y = cur[42 + vy];
            Y = w4_add(Y, cur[86 + vy]);
            const cx<R> ab = -Jb[1] + Jb[2] + -Jb[3] + Jb[4];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<6u, false>(Yb, curb, 42 + vy, lane, act);
              } else {
                curb.atomic_add(42 + vy, Yb);
              }
              if (full) {
                w4_warp_reduce_add<6u, false>(Yb, curb, 86 + vy, lane, act);
              } else {
                curb.atomic_add(86 + vy, Yb);
              }
            }
          }
          {
            const int vy = vt[608];
            W4<R> Y = cur[50 + vy];
            Y = w4_sub(Y, cur[70 + vy]);
            const cx<R> ab = Jb[0] + -Jb[1] + -Jb[3] + Jb[5];
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<6u, false>(Yb, curb, 50 + vy, lane, act);
              } else {
                curb.atomic_add(50 + vy, Yb);
              }
              if (full) {
                w4_warp_reduce_add<6u, false>(w4_neg(Yb), curb, 70 + vy, lane, act);
              } else {
                curb.atomic_add(70 + vy, w4_neg(Yb));
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<25u, false>(Xb, xbb, 72 + vx, lane, act);
            } else {
              xbb.atomic_add(72 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[224];
          const W4<R> X = xb[76 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[768];
            W4<R> Y = cur[18 + vy];
            const cx<R> ab = mul_i(Jb[0]) + mul_mi(Jb[2]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<28u, false>(Yb, curb, 18 + vy, lane, act);
              } else {
                curb.atomic_add(18 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<3u, false>(Xb, xbb, 76 + vx, lane, act);
            } else {
              xbb.atomic_add(76 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[672];
          const W4<R> X = xb[84 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[320];
            W4<R> Y = cur[14 + vy];
            const cx<R> ab = mul_i(Jb[1]) + mul_mi(Jb[4]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<21u, false>(Yb, curb, 14 + vy, lane, act);
              } else {
                curb.atomic_add(14 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<10u, false>(Xb, xbb, 84 + vx, lane, act);
            } else {
              xbb.atomic_add(84 + vx, Xb);
            }
          }
        }
        {
          const int vx = vt[704];
          const W4<R> X = xb[92 + vx];
          W4<R> Xb = w4_zero<R>();
          {
            const int vy = vt[288];
            W4<R> Y = cur[10 + vy];
            const cx<R> ab = mul_i(Jb[3]) + mul_mi(Jb[5]);
            if constexpr ((PASS & 2) != 0) w4_acc_conj(Xb, Y, ab);
            if constexpr ((PASS & 1) != 0) {
              const W4<R> Yb = w4_conj_scale(X, ab);
              if (full) {
                w4_warp_reduce_add<13u, false>(Yb, curb, 10 + vy, lane, act);
              } else {
                curb.atomic_add(10 + vy, Yb);
              }
            }
          }
          if constexpr ((PASS & 2) != 0) {
            if (full) {
              w4_warp_reduce_add<18u, false>(Xb, xbb, 92 + vx, lane, act);
            } else {
              xbb.atomic_add(92 + vx, Xb);
            }
          }
        }
      } break;
      default: break;
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
    constexpr int t[NMOM][3] = {{0, 1, 0}, {0, 2, 0}, {0, 4, 0}, {0, 8, 0}, {0, 16, 0}, {1, 19, 3}, {1, 2, 2}, {1, 16, 0}, {1, 18, 2}, {1, 1, 1}, {1, 5, 1}, {1, 22, 2}, {1, 7, 3}, {1, 21, 1}, {1, 3, 3}, {1, 20, 0}, {1, 17, 1}, {1, 6, 2}, {1, 22, 20}, {1, 21, 20}, {1, 7, 4}};
    return t[j][k];
  }
  // propagators: {momentum entry, 0 gluon / 1 top / 2 photon / 3 Z}
  static __host__ __device__ constexpr int prop(int j, int k) {
    constexpr int t[NPROP][2] = {{5, 0}, {8, 0}, {10, 1}, {11, 1}, {12, 1}, {13, 1}, {14, 0}, {15, 1}, {16, 0}, {17, 1}};
    return t[j][k];
  }
  // propagator entries formed from each momentum entry (-1: none)
  static __host__ __device__ constexpr int mom_prop(int j, int k) {
    constexpr int t[NMOM][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {0, -1}, {-1, -1}, {-1, -1}, {1, -1}, {-1, -1}, {2, -1}, {3, -1}, {4, -1}, {5, -1}, {6, -1}, {7, -1}, {8, -1}, {9, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
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
