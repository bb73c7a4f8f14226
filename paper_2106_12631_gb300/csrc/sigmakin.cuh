// Per-event squared matrix elements (the paper's SIGMAKIN, Sec. 4 and
// Fig. 6): one thread per (event, good helicity).
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
//   3. colour sum |M_h|^2 = J^dagger C J / den (Sec. 2).
//   4. helicity sum per event in a fixed order (bitwise reproducible), FP64.
// The helicity list comes from the device mask written by the filtering pass
// (Sec. 2: "pre-determines which helicity combinations are allowed").
#pragma once
#include "process.cuh"

namespace mg {

constexpr int kSigmaThreads = 128;

template <class P>
struct SigCfg {
  static constexpr int NT = kSigmaThreads;
  static constexpr int EVMIN = (NT / P::NHEL) > 0 ? (NT / P::NHEL) : 1;  // all helicities good
  static constexpr int EVCAP = (4 * EVMIN) < 32 ? 4 * EVMIN : 32;
};

struct SigArgs {
  int64_t nevt;
  const double* __restrict__ mom;  // [npar][4][nevt]
  const int32_t* __restrict__ mask;  // [nhel] 0/1 (sum mode)
  double* __restrict__ me;           // [nevt] (sum mode)
  int32_t* __restrict__ mask_out;    // [nhel] (filter mode, pre-zeroed)
  PhysParams pp;
};

// |M_h|^2 summed over colours, CUDA cores.  C = CNUM / CDEN, real symmetric.
template <class P, class R>
__device__ __forceinline__ R colour_sum_simt(const cx<R>* J) {
  R s = R(0);
#pragma unroll
  for (int i = 0; i < P::NCOLOR; ++i) {
    R tr = R(0), ti = R(0);
#pragma unroll
    for (int j = 0; j < P::NCOLOR; ++j) {
      if (P::cnum(i, j) == 0) continue;
      tr += R(P::cnum(i, j)) * J[j].re;
      ti += R(P::cnum(i, j)) * J[j].im;
    }
    s += J[i].re * tr + J[i].im * ti;
  }
  return s / R(P::CDEN);
}

template <class P, class R>
struct SigShared {
  static constexpr int EVCAP = SigCfg<P>::EVCAP;
  double p[EVCAP][P::NPAR][4];
  R K[EVCAP][P::NMOM][4];
  cx<R> prop[EVCAP][P::NPROP];
  int mom_tab[P::NMOM][3];
  int prop_tab[P::NPROP][2];
  int good[P::NHEL];
  int ngood;
  double m2[kSigmaThreads];
};

// Phase 1: per-event tables.  Returns the number of events of this CTA.
template <class P, class R>
__device__ __forceinline__ void event_tables(SigShared<P, R>& sh, const SigArgs& a, int64_t e0, int nev) {
  const int tid = threadIdx.x;
  for (int t = tid; t < nev * P::NPAR * 4; t += blockDim.x) {
    const int e = t % nev, c = t / nev;
    sh.p[e][c >> 2][c & 3] = a.mom[(int64_t)c * a.nevt + e0 + e];
  }
  __syncthreads();
  for (int t = tid; t < nev * (P::NMOM + P::NPROP); t += blockDim.x) {
    const int e = t % nev, j = t / nev;
    const int mj = j < P::NMOM ? j : sh.prop_tab[j - P::NMOM][0];
    const int kind = sh.mom_tab[mj][0], lmask = sh.mom_tab[mj][1], smask = sh.mom_tab[mj][2];
    double k[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l = 0; l < P::NPAR; ++l) {
      if (!(lmask >> l & 1)) continue;
      const double sg = (kind == 1 && (smask >> l & 1)) ? -1.0 : 1.0;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) k[mu] += sg * sh.p[e][l][mu];
    }
    if (j < P::NMOM) {
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) sh.K[e][j][mu] = R(k[mu]);
    } else {
      double re, im;
      propagator_fp64(k, sh.prop_tab[j - P::NMOM][1], a.pp, re, im);
      sh.prop[e][j - P::NMOM] = cx<R>(R(re), R(im));
    }
  }
  __syncthreads();
}

template <class P, class R>
__device__ __forceinline__ void load_tables(SigShared<P, R>& sh) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < P::NMOM; ++j) {
      sh.mom_tab[j][0] = P::mom(j, 0); sh.mom_tab[j][1] = P::mom(j, 1); sh.mom_tab[j][2] = P::mom(j, 2);
    }
#pragma unroll
    for (int j = 0; j < P::NPROP; ++j) { sh.prop_tab[j][0] = P::prop(j, 0); sh.prop_tab[j][1] = P::prop(j, 1); }
  }
}

template <class P>
__device__ __forceinline__ void decode_helicity(int ihel, int* hel) {
#pragma unroll
  for (int k = 0; k < P::NPAR; ++k) hel[k] = ((ihel >> (P::NPAR - 1 - k)) & 1) ? 1 : -1;
}

// Helicity-summed matrix elements.  R = double: plain FP64 path; R = float:
// mixed path with the colour sum on CUDA cores in FP32.
template <class P, class R>
__global__ void __launch_bounds__(kSigmaThreads) sigmakin_kernel(SigArgs a, Couplings<R> cp) {
  __shared__ SigShared<P, R> sh;
  const int tid = threadIdx.x;
  load_tables<P, R>(sh);
  if (tid == 0) {
    int n = 0;
    for (int h = 0; h < P::NHEL; ++h)
      if (a.mask[h]) sh.good[n++] = h;
    sh.ngood = n;
  }
  __syncthreads();
  const int ng = sh.ngood;
  const int ev = ng > 0 ? min(SigCfg<P>::EVCAP, (int)blockDim.x / ng) : SigCfg<P>::EVMIN;
  const int64_t e0 = (int64_t)blockIdx.x * ev;
  if (e0 >= a.nevt) return;
  const int nev = (int)min((int64_t)ev, a.nevt - e0);
  if (ng == 0) {
    if (tid < nev) a.me[e0 + tid] = 0.0;
    return;
  }
  event_tables<P, R>(sh, a, e0, nev);
  const int e = tid / ng, h = tid - e * ng;
  double m2 = 0.0;
  if (e < nev) {
    int hel[P::NPAR];
    decode_helicity<P>(sh.good[h], hel);
    cx<R> J[P::NCOLOR];
    P::template amplitudes<R>(&sh.K[e][0][0], sh.prop[e], hel, cp, J);
    m2 = (double)colour_sum_simt<P, R>(J);
  }
  sh.m2[tid] = m2;
  __syncthreads();
  if (tid < nev) {
    double s = 0.0;
    for (int k = 0; k < ng; ++k) s += sh.m2[tid * ng + k];
    a.me[e0 + tid] = s * P::NORM;
  }
}

// Helicity filtering (FP64): every helicity of the first nevt events; a
// helicity is kept if any event gives a non-zero |M_h|^2.
template <class P>
__global__ void __launch_bounds__(kSigmaThreads) filter_kernel(SigArgs a, Couplings<double> cp) {
  __shared__ SigShared<P, double> sh;
  const int tid = threadIdx.x;
  load_tables<P, double>(sh);
  __syncthreads();
  constexpr int ev = SigCfg<P>::EVMIN;
  const int64_t e0 = (int64_t)blockIdx.x * ev;
  if (e0 >= a.nevt) return;
  const int nev = (int)min((int64_t)ev, a.nevt - e0);
  event_tables<P, double>(sh, a, e0, nev);
  const int e = tid / P::NHEL, h = tid % P::NHEL;
  if (e < nev) {
    int hel[P::NPAR];
    decode_helicity<P>(h, hel);
    cx<double> J[P::NCOLOR];
    P::template amplitudes<double>(&sh.K[e][0][0], sh.prop[e], hel, cp, J);
    const double m2 = colour_sum_simt<P, double>(J);
    if (m2 != 0.0) atomicOr(a.mask_out + h, 1);
  }
}

}  // namespace mg
