// Gradient of the squared matrix element with respect to the random numbers
// (not in the paper): d me / d rnd for every event, through RAMBO and the
// helicity amplitudes, by a hand-written adjoint.
//
// One thread per (event, good helicity), as in SIGMAKIN.  Per CTA:
//   1. RAMBO forward (FP64) for the CTA's events from their random numbers;
//   2. per-event momentum sums and propagator factors (FP64 -> R);
//   3. every thread recomputes its helicity's diagram program and runs its
//      adjoint (generated amplitudes_grad): d|M_h|^2 / d(final momenta) in R —
//      the recomputation per helicity replaces storing any current;
//   4. fixed-order FP64 sum over helicities, times the averaging factor and
//      the incoming gradient dL/dme;
//   5. RAMBO adjoint (FP64) -> dL/d rnd; rows RAMBO does not consume get 0.
#pragma once
#include "helas_adj.cuh"
#include "launch.h"
#include "rambo.cuh"
#include "sigmakin.cuh"

namespace mg {

struct GradArgs {
  int64_t nevt;
  double ecm;
  const double* __restrict__ rnd;   // [nrows][nevt]
  int nrows;
  const int32_t* __restrict__ mask;
  const double* __restrict__ gout;  // [nevt] or null (= 1)
  double* __restrict__ grad;        // [nrows][nevt]
  double* __restrict__ me;          // [nevt] or null
  PhysParams pp;
  RamboSetup st;
};

template <class P, class R>
struct GradLayout {
  using S = SigLayout<P, R, CS_SIMT>;
  using C = SigCfg<P>;
  static constexpr int NF = P::NFINAL;
  static constexpr size_t o_r = align_up(S::bytes, 16);                       // double [EVCAP][4 NF]
  static constexpr size_t o_pb = align_up(o_r + 8 * C::EVCAP * 4 * NF, 16);  // double [NT][4 NF]
  static constexpr size_t bytes = o_pb + 8 * C::NT * 4 * NF;
};

template <class P, class R>
__global__ void __launch_bounds__(SigCfg<P>::NT, 1) sigmakin_grad_kernel(GradArgs a, Couplings<R> cp) {
  using C = SigCfg<P>;
  using L = SigLayout<P, R, CS_SIMT>;
  using G = GradLayout<P, R>;
  constexpr int NF = P::NFINAL;
  extern __shared__ __align__(1024) unsigned char smem[];
  int* good = reinterpret_cast<int*>(smem + L::o_good);
  int* misc = reinterpret_cast<int*>(smem + L::o_misc);
  double* sm2 = reinterpret_cast<double*>(smem + L::o_m2);
  auto sr = reinterpret_cast<double(*)[4 * NF]>(smem + G::o_r);
  auto spb = reinterpret_cast<double(*)[4 * NF]>(smem + G::o_pb);
  auto p = reinterpret_cast<double(*)[P::NPAR][4]>(smem + L::o_p);
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
  // 1. RAMBO forward per event
  if (tid < nev) {
    double r[4 * NF];
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) { r[k] = a.rnd[(int64_t)k * a.nevt + e0 + tid]; sr[tid][k] = r[k]; }
    RamboState<NF> z;
    rambo_forward<NF>(r, a.ecm, a.st, z);
    const double h = 0.5 * a.ecm;
    p[tid][0][0] = h; p[tid][0][1] = 0.0; p[tid][0][2] = 0.0; p[tid][0][3] = h;
    p[tid][1][0] = h; p[tid][1][1] = 0.0; p[tid][1][2] = 0.0; p[tid][1][3] = -h;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) p[tid][2 + f][mu] = z.k[f][mu];
  }
  __syncthreads();
  // 2. tables
  build_tables<P, R, L>(smem, a.pp, nev);
  // 3. forward + adjoint of this thread's helicity
  const bool active = ng > 0 && tid < nev * ng;
  double m2 = 0.0;
  double pbl[4 * NF];
#pragma unroll
  for (int k = 0; k < 4 * NF; ++k) pbl[k] = 0.0;
  if (active) {
    const int e = tid / ng, h = tid - e * ng;
    int hel[P::NPAR];
    decode_helicity<P>(good[h], hel);
    const R* K = reinterpret_cast<const R*>(smem + L::o_K) + e * P::NMOM * 4;
    const cx<R>* pr = reinterpret_cast<const cx<R>*>(smem + L::o_pr) + e * P::NPROP;
    R pb[4 * P::NPAR];
#pragma unroll
    for (int k = 0; k < 4 * P::NPAR; ++k) pb[k] = R(0);
    m2 = (double)P::template amplitudes_grad<R>(K, pr, hel, cp, pb);
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) pbl[k] = (double)pb[8 + k];
  }
  sm2[tid] = m2;
#pragma unroll
  for (int k = 0; k < 4 * NF; ++k) spb[tid][k] = pbl[k];
  __syncthreads();
  // 4.-5. helicity sum, RAMBO adjoint
  if (tid < nev) {
    const int64_t i = e0 + tid;
    double me = 0.0, kb[NF][4];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) kb[f][mu] = 0.0;
    for (int k = 0; k < ng; ++k) {
      const int t = tid * ng + k;
      me += sm2[t];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) kb[f][mu] += spb[t][4 * f + mu];
    }
    const double g = (a.gout ? a.gout[i] : 1.0) * P::NORM;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) kb[f][mu] *= g;
    double r[4 * NF], rb[4 * NF];
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) r[k] = sr[tid][k];
    RamboState<NF> z;
    rambo_forward<NF>(r, a.ecm, a.st, z);
    rambo_adjoint<NF>(r, a.ecm, a.st, z, kb, rb);
    for (int k = 0; k < a.nrows; ++k) a.grad[(int64_t)k * a.nevt + i] = k < 4 * NF ? rb[k] : 0.0;
    if (a.me) a.me[i] = me * P::NORM;
  }
}

template <class P, class R>
cudaError_t launch_grad_variant(const GradArgs& a, const Couplings<R>& cp, cudaStream_t s) {
  using G = GradLayout<P, R>;
  const int64_t grid = (a.nevt + SigCfg<P>::EVMIN - 1) / SigCfg<P>::EVMIN;
  if (grid == 0) return cudaSuccess;
  auto k = sigmakin_grad_kernel<P, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, SigCfg<P>::NT, G::bytes, s>>>(a, cp);
  return cudaGetLastError();
}

}  // namespace mg
