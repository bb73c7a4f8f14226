// Per-event squared matrix elements (the paper's SIGMAKIN, Sec. 4): one
// thread per (event, good helicity).
//
// A CTA of NT threads handles EV consecutive events x ngood helicities
// (EV = min(EVCAP, NT / ngood)).  Phases:
//   1. external momenta of the CTA's events -> shared memory (FP64);
//      per event: every outgoing momentum sum the diagram program needs and
//      every propagator factor, formed in FP64 (both modes) -> shared memory
//      in the working precision R.  These are helicity independent, so they
//      are computed once per event instead of once per helicity.
//   2. each thread runs the straight-line diagram program of its helicity:
//      external wavefunctions, currents, amplitudes -> dual amplitudes J.
//      FP64 keeps J in registers; FP32 accumulates J in shared memory and
//      re-aligns the CTA's warps every few routine calls so that they stream
//      through the (large) program together and share instruction-cache lines.
//   3. colour sum |M_h|^2 = J^dagger C J / den (Sec. 2) on CUDA cores or on the
//      tensor cores (colour_tc.cuh).
//   4. helicity sum per event in a fixed order (bitwise reproducible), FP64.
// The helicity list comes from the device mask written by the filtering pass
// (Sec. 2: helicity combinations with a non-zero contribution are determined
// on a small set of events first).
#pragma once
#include <cuda_bf16.h>

#include "colour_tc.cuh"
#include "process.cuh"
#include "rambo.cuh"

namespace mg {

enum ColourSum { CS_SIMT = 0, CS_TC = 1 };

template <class P>
struct SigCfg {
  static constexpr int NT = P::NCOLOR >= 6 ? 256 : 128;
  static constexpr int EVMIN = (NT / P::NHEL) > 0 ? (NT / P::NHEL) : 1;  // all helicities good
  static constexpr int EVCAP = (4 * EVMIN) < 32 ? 4 * EVMIN : 32;
  static constexpr int KP = ((P::NCOLOR + 15) / 16) * 16;  // colour flows padded to the MMA K step
  static constexpr int NP = KP;                            // ... and to a valid MMA N (M = 128)
  static constexpr int MBLK = NT / 128;                    // 128-row MMA blocks per CTA
};

struct SigArgs {
  int64_t nevt;
  const double* __restrict__ mom;     // [npar][4][nevt]
  const int32_t* __restrict__ mask;   // [nhel] 0/1 (sum mode)
  double* __restrict__ me;            // [nevt] (sum mode)
  int32_t* __restrict__ mask_out;     // [nhel] (filter mode, pre-zeroed)
  PhysParams pp;
  const double* __restrict__ hel_rnd;  // [nevt] uniforms for the helicity choice, or null
  int32_t* __restrict__ hel_out;       // [nevt] chosen helicity (-1 if me = 0), or null
  const double* __restrict__ col_rnd;  // [nevt] uniforms for the colour-flow choice, or null
  int32_t* __restrict__ col_out;       // [nevt] chosen colour flow (-1 if me = 0), or null
};

// RAMBO inside the SIGMAKIN kernel (the fused entry points), a kernel argument
// of its own so that the other kernels' arguments stay as they are: the
// uniforms of event i, row k from rnd[k][nevt], or (rnd == nullptr) from the
// counter-based generator at (key, first_event + i, k); wgt[nevt] receives
// RAMBO's weight.
struct RamboArgs {
  const double* __restrict__ rnd;
  double* __restrict__ wgt;
  double ecm;
  uint64_t key;
  int64_t first_event;
  RamboSetup st;
};

// ---- dual-amplitude accumulators ------------------------------------------------
template <class R, int NC>
struct RegAcc {
  cx<R> j[NC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int s = 0; s < NC; ++s) j[s] = cx<R>(R(0), R(0));
  }
  __device__ __forceinline__ void add(int s, cx<R> a) { j[s] += a; }
  __device__ __forceinline__ void sub(int s, cx<R> a) { j[s] -= a; }
  __device__ __forceinline__ void addi(int s, cx<R> a) { j[s] += mul_i(a); }
  __device__ __forceinline__ void subi(int s, cx<R> a) { j[s] -= mul_i(a); }
};
// FP32 J in shared memory, [2][NC][NT] floats, this thread's column pre-offset
template <int NC, int NT>
struct SmemAcc {
  float* j;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int s = 0; s < 2 * NC; ++s) j[s * NT] = 0.0f;
  }
  __device__ __forceinline__ void add(int s, cx<float> a) { j[s * NT] += a.re; j[(NC + s) * NT] += a.im; }
  __device__ __forceinline__ void sub(int s, cx<float> a) { j[s * NT] -= a.re; j[(NC + s) * NT] -= a.im; }
  __device__ __forceinline__ void addi(int s, cx<float> a) { j[s * NT] -= a.im; j[(NC + s) * NT] += a.re; }
  __device__ __forceinline__ void subi(int s, cx<float> a) { j[s * NT] += a.im; j[(NC + s) * NT] -= a.re; }
};
struct NoSync {
  static __device__ __forceinline__ void sync() {}
};
struct CtaSync {
  static __device__ __forceinline__ void sync() { __syncthreads(); }
};

// |M_h|^2 summed over colours on CUDA cores.  C = cnum / CDEN, real symmetric.
template <class P, class R, class GetRe, class GetIm>
__device__ __forceinline__ R colour_sum_simt(GetRe jre, GetIm jim) {
  R re[P::NCOLOR], im[P::NCOLOR];
#pragma unroll
  for (int s = 0; s < P::NCOLOR; ++s) { re[s] = jre(s); im[s] = jim(s); }
  R sum = R(0);
#pragma unroll
  for (int i = 0; i < P::NCOLOR; ++i) {
    R tr = R(0), ti = R(0);
#pragma unroll
    for (int j = 0; j < P::NCOLOR; ++j) {
      if (P::cnum(i, j) == 0) continue;
      tr += R(P::cnum(i, j)) * re[j];
      ti += R(P::cnum(i, j)) * im[j];
    }
    sum += re[i] * tr + im[i] * ti;
  }
  return sum / R(P::CDEN);
}

// ---- shared-memory layout ---------------------------------------------------------
__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <class P, class R, int CS>
struct SigLayout {
  using C = SigCfg<P>;
  static constexpr bool SMEMJ = sizeof(R) == 4;
  static constexpr bool TC = CS == CS_TC;
  static constexpr size_t o_momtab = 0;
  static constexpr size_t o_proptab = align_up(o_momtab + 12 * P::NMOM, 16);
  static constexpr size_t o_good = align_up(o_proptab + 8 * P::NPROP, 16);
  static constexpr size_t o_misc = align_up(o_good + 4 * P::NHEL, 16);  // ngood, tmem base, mbarrier
  static constexpr size_t o_p = align_up(o_misc + 32, 16);
  static constexpr size_t o_K = align_up(o_p + 8 * C::EVCAP * P::NPAR * 4, 16);
  static constexpr size_t o_pr = align_up(o_K + sizeof(R) * C::EVCAP * P::NMOM * 4, 16);
  static constexpr size_t o_m2 = align_up(o_pr + 2 * sizeof(R) * C::EVCAP * P::NPROP, 16);
  static constexpr size_t o_J = align_up(o_m2 + 8 * C::NT, 128);
  static constexpr size_t o_A = align_up(o_J + (SMEMJ ? 8 * P::NCOLOR * C::NT : 0), 1024);
  static constexpr size_t tileA = 128 * C::KP * 2;  // one 128-row BF16 tile
  static constexpr size_t o_B = o_A + (TC ? 3 * 2 * C::MBLK * tileA : 0);
  static constexpr size_t bytes = o_B + (TC ? C::NP * C::KP * 2 : 0);
  static constexpr uint32_t TMEM_COLS = tc::tmem_cols(C::MBLK * 2 * C::NP);
  static_assert(TMEM_COLS <= 512, "TMEM holds 512 columns");
};

// Phase 1b: per-event tables from the FP64 momenta already in shared memory.
template <class P, class R, class L, int NTS = SigCfg<P>::NT>
__device__ __forceinline__ void build_tables(unsigned char* smem, const PhysParams& pp, int nev) {
  const int tid = threadIdx.x;
  auto p = reinterpret_cast<double(*)[P::NPAR][4]>(smem + L::o_p);
  auto K = reinterpret_cast<R(*)[P::NMOM][4]>(smem + L::o_K);
  auto pr = reinterpret_cast<cx<R>(*)[P::NPROP]>(smem + L::o_pr);
  const int(*mom_tab)[3] = reinterpret_cast<const int(*)[3]>(smem + L::o_momtab);
  const int(*prop_tab)[2] = reinterpret_cast<const int(*)[2]>(smem + L::o_proptab);
  for (int t = tid; t < nev * (P::NMOM + P::NPROP); t += NTS) {
    const int e = t % nev, j = t / nev;
    const int mj = j < P::NMOM ? j : prop_tab[j - P::NMOM][0];
    const int kind = mom_tab[mj][0], lmask = mom_tab[mj][1], smask = mom_tab[mj][2];
    double k[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l = 0; l < P::NPAR; ++l) {
      if (!(lmask >> l & 1)) continue;
      const double sg = (kind == 1 && (smask >> l & 1)) ? -1.0 : 1.0;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) k[mu] += sg * p[e][l][mu];
    }
    if (j < P::NMOM) {
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) K[e][j][mu] = R(k[mu]);
    } else {
      double re, im;
      propagator_fp64(k, prop_tab[j - P::NMOM][1], pp, re, im);
      pr[e][j - P::NMOM] = cx<R>(R(re), R(im));
    }
  }
  __syncthreads();
}

// Phase 1: external momenta (global -> shared) and the per-event tables
// (NTS threads).
template <class P, class R, class L, int NTS = SigCfg<P>::NT>
__device__ __forceinline__ void event_tables(unsigned char* smem, const SigArgs& a, int64_t e0, int nev) {
  const int tid = threadIdx.x;
  auto p = reinterpret_cast<double(*)[P::NPAR][4]>(smem + L::o_p);
  for (int t = tid; t < nev * P::NPAR * 4; t += NTS) {
    const int e = t % nev, c = t / nev;
    p[e][c >> 2][c & 3] = a.mom[(int64_t)c * a.nevt + e0 + e];
  }
  __syncthreads();
  build_tables<P, R, L, NTS>(smem, a.pp, nev);
}

template <class P, class L>
__device__ __forceinline__ void load_tables(unsigned char* smem) {
  if (threadIdx.x == 0) {
    int(*mom_tab)[3] = reinterpret_cast<int(*)[3]>(smem + L::o_momtab);
    int(*prop_tab)[2] = reinterpret_cast<int(*)[2]>(smem + L::o_proptab);
#pragma unroll
    for (int j = 0; j < P::NMOM; ++j) {
      mom_tab[j][0] = P::mom(j, 0); mom_tab[j][1] = P::mom(j, 1); mom_tab[j][2] = P::mom(j, 2);
    }
#pragma unroll
    for (int j = 0; j < P::NPROP; ++j) { prop_tab[j][0] = P::prop(j, 0); prop_tab[j][1] = P::prop(j, 1); }
  }
}

template <class P>
__device__ __forceinline__ void decode_helicity(int ihel, int* hel) {
#pragma unroll
  for (int k = 0; k < P::NPAR; ++k) hel[k] = ((ihel >> (P::NPAR - 1 - k)) & 1) ? 1 : -1;
}

// ---- tensor-core colour sum of the CTA's NT rows ---------------------------------
// J: [2][NC][NT] FP32 in shared memory.  Returns |M_h|^2 of this thread's row
// (NaN if the MMA did not complete within the wait limit).
template <class P, class L>
__device__ __forceinline__ float colour_sum_tc(unsigned char* smem, const float* J, uint32_t tmem, uint32_t mbar) {
  using C = SigCfg<P>;
  constexpr int NC = P::NCOLOR, KP = C::KP, NT = C::NT;
  const int tid = threadIdx.x;
  const int b = tid >> 7, r = tid & 127;
  // 1. three BF16 terms of this thread's row, re and im, in the canonical layout
#pragma unroll
  for (int c = 0; c < 2; ++c) {
#pragma unroll
    for (int k0 = 0; k0 < KP; k0 += 8) {
      uint32_t w[3][4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        uint16_t hb[3][2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k = k0 + q + u;
          const float x = k < NC ? J[(c * NC + k) * NT + tid] : 0.0f;
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
        unsigned char* tile = smem + L::o_A + ((sp * 2 + c) * C::MBLK + b) * L::tileA;
        *reinterpret_cast<uint4*>(tile + tc::kmajor_offset<KP>(r, k0)) = make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
      }
    }
  }
  tc::fence_async_shared();
  __syncthreads();
  // 2. one thread issues the MMAs: D[b][c] (+)= A[split][c][b] x B over K steps
  if (tid == 0) {
    tc::fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_bf16(128, C::NP);
    constexpr uint32_t LBO = 128, SBO = (KP / 8) * 128;
    const uint32_t bbase = tc::smem_addr(smem + L::o_B);
#pragma unroll
    for (int bb = 0; bb < C::MBLK; ++bb)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const uint32_t d = tmem + (uint32_t)((bb * 2 + c) * C::NP);
#pragma unroll
        for (int sp = 0; sp < 3; ++sp) {
          const uint32_t abase = tc::smem_addr(smem + L::o_A + ((sp * 2 + c) * C::MBLK + bb) * L::tileA);
#pragma unroll
          for (int j = 0; j < KP / 16; ++j)
            tc::mma_bf16(d, tc::smem_desc(abase + j * 256, LBO, SBO), tc::smem_desc(bbase + j * 256, LBO, SBO),
                         idesc, (sp | j) != 0);
        }
      }
    tc::mma_commit(mbar);
  }
  const bool ok = tc::mbar_wait(mbar, 0);
  tc::fence_after_sync();
  // 3. read this warp's 32 rows back (lanes 32 (warp % 4) .. +31 of block b)
  const int warp = tid >> 5;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  float yr[C::NP], yi[C::NP];
#pragma unroll
  for (int c0 = 0; c0 < C::NP; c0 += 16) {
    tc::tmem_ld16(tmem + lane_base + (uint32_t)((b * 2 + 0) * C::NP + c0), yr + c0);
    tc::tmem_ld16(tmem + lane_base + (uint32_t)((b * 2 + 1) * C::NP + c0), yi + c0);
  }
  tc::tmem_wait_ld();
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < NC; ++k) s += J[k * NT + tid] * yr[k] + J[(NC + k) * NT + tid] * yi[k];
  s *= 1.0f / (float)P::CDEN;
  if (!ok) {
    tc::mbar_wait(mbar, 0);  // second bounded wait for the MMAs still in flight
    s = __int_as_float(0x7fc00000);
  }
  return s;
}

// Helicity-summed matrix elements.  R = double: FP64 path.  R = float: mixed
// path, colour sum on CUDA cores (CS_SIMT) or tensor cores (CS_TC).
template <class P, class R, int CS>
__global__ void __launch_bounds__(SigCfg<P>::NT, 1) sigmakin_kernel(SigArgs a, Couplings<R> cp) {
  using C = SigCfg<P>;
  using L = SigLayout<P, R, CS>;
  extern __shared__ __align__(1024) unsigned char smem[];
  int* good = reinterpret_cast<int*>(smem + L::o_good);
  int* misc = reinterpret_cast<int*>(smem + L::o_misc);
  double* sm2 = reinterpret_cast<double*>(smem + L::o_m2);
  const int tid = threadIdx.x;
  load_tables<P, L>(smem);
  if (tid == 0) {
    int n = 0;
    for (int h = 0; h < P::NHEL; ++h)
      if (a.mask[h]) good[n++] = h;
    misc[0] = n;
  }
  __syncthreads();
  const int ng = misc[0];
  const int ev = ng > 0 ? min(C::EVCAP, C::NT / ng) : C::EVMIN;
  const int64_t e0 = (int64_t)blockIdx.x * ev;
  if (e0 >= a.nevt) return;
  const int nev = (int)min((int64_t)ev, a.nevt - e0);
  if (ng == 0) {
    if (tid < nev) a.me[e0 + tid] = 0.0;
    return;
  }
  uint32_t tmem = 0, mbar = 0;
  if constexpr (L::TC) {
    // tensor memory for the accumulators, the MMA completion barrier, and the
    // colour matrix numerators (BF16, canonical layout) for the B operand
    if (tid < 32) tc::tmem_alloc(tc::smem_addr(misc + 1), L::TMEM_COLS);
    mbar = tc::smem_addr(misc + 4);
    if (tid == 0) tc::mbar_init(mbar, 1);
    const uint4* src = reinterpret_cast<const uint4*>(P::colour_bf16_image());
    uint4* dst = reinterpret_cast<uint4*>(smem + L::o_B);
    for (int i = tid; i < C::NP * C::KP * 2 / 16; i += C::NT) dst[i] = src[i];
    tc::fence_async_shared();
    tc::fence_before_sync();
  }
  event_tables<P, R, L>(smem, a, e0, nev);  // ends with __syncthreads()
  if constexpr (L::TC) {
    tc::fence_after_sync();
    tmem = static_cast<uint32_t>(misc[1]);
  }
  const bool active = tid < nev * ng;
  const int e = active ? tid / ng : 0;
  const int h = active ? tid - e * ng : 0;
  int hel[P::NPAR];
  decode_helicity<P>(good[h], hel);
  const R* K = reinterpret_cast<const R*>(smem + L::o_K) + e * P::NMOM * 4;
  const cx<R>* pr = reinterpret_cast<const cx<R>*>(smem + L::o_pr) + e * P::NPROP;
  double m2;
  if constexpr (sizeof(R) == 8) {
    RegAcc<R, P::NCOLOR> J;
    P::template amplitudes<R, RegAcc<R, P::NCOLOR>, NoSync>(K, pr, hel, cp, J);
    m2 = colour_sum_simt<P, R>([&](int s) { return J.j[s].re; }, [&](int s) { return J.j[s].im; });
  } else {
    float* Js = reinterpret_cast<float*>(smem + L::o_J);
    SmemAcc<P::NCOLOR, C::NT> J{Js + tid};
    P::template amplitudes<float, SmemAcc<P::NCOLOR, C::NT>, CtaSync>(K, pr, hel, cp, J);
    if constexpr (L::TC) {
      __syncthreads();
      m2 = (double)colour_sum_tc<P, L>(smem, Js, tmem, mbar);
    } else {
      m2 = (double)colour_sum_simt<P, float>([&](int s) { return Js[s * C::NT + tid]; },
                                             [&](int s) { return Js[(P::NCOLOR + s) * C::NT + tid]; });
    }
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
    double s = 0.0;
    for (int k = 0; k < ng; ++k) s += sm2[tid * ng + k];
    a.me[e0 + tid] = s * P::NORM;
  }
}

// Helicity filtering (FP64): every helicity of the first nevt events; a
// helicity is kept if any event gives a non-zero |M_h|^2.
// Helicity filter: helicity h is kept if |M_h|^2 != 0 for any of the filter
// events (FP64, the straight-line program of each helicity).  One thread per
// (event, helicity) in CTAs of FILTER_NT threads, so that the few filter
// events spread over many SMs (each thread's FP64 program is long).
constexpr int FILTER_NT = 16;
template <class P>
__global__ void __launch_bounds__(FILTER_NT) filter_kernel(SigArgs a, Couplings<double> cp) {
  using L = SigLayout<P, double, CS_SIMT>;
  constexpr int HB = (P::NHEL + FILTER_NT - 1) / FILTER_NT;  // helicity blocks per event
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)(blockIdx.x / HB);
  const int h = (int)(blockIdx.x % HB) * FILTER_NT + tid;
  if (e0 >= a.nevt) return;
  load_tables<P, L>(smem);
  __syncthreads();
  event_tables<P, double, L, FILTER_NT>(smem, a, e0, 1);
  if (h < P::NHEL) {
    int hel[P::NPAR];
    decode_helicity<P>(h, hel);
    const double* K = reinterpret_cast<const double*>(smem + L::o_K);
    const cx<double>* pr = reinterpret_cast<const cx<double>*>(smem + L::o_pr);
    RegAcc<double, P::NCOLOR> J;
    P::template amplitudes<double, RegAcc<double, P::NCOLOR>, NoSync>(K, pr, hel, cp, J);
    const double m2 =
        colour_sum_simt<P, double>([&](int s) { return J.j[s].re; }, [&](int s) { return J.j[s].im; });
    if (m2 != 0.0) atomicOr(a.mask_out + h, 1);
  }
}

}  // namespace mg
