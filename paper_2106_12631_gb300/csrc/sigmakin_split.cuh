// Kernel-split variant of the helicity-shared program (the outlook of
// Sec. 4: SIGMAKIN split into smaller kernels orchestrated with CUDA Graphs,
// to relieve the one large kernel).  Two kernels per chunk of events:
//   currents:   momenta -> tables -> external wavefunctions -> every current
//               variant (phases 1-2 of the helicity-shared kernel), written
//               as one record per event (HsRecord) to a chunk buffer;
//   amplitudes: the records back into shared memory, then phases 3-5 of the
//               helicity-shared kernel (amputated currents, contractions,
//               colour sum on CUDA cores, helicity sum, choices).
// Chunks small enough that two chunk buffers stay in L2 alternate, so that the
// currents of chunk c + 1 run beside the amplitudes of chunk c; the launches
// of a whole batch are captured once into a CUDA graph (split_graph.cu).
#pragma once
#include <cstring>

#include "launch.h"
#include "sigmakin_hs.cuh"

namespace mg {

// the currents kernel's own smaller CTA: 4 events, 128 threads, three CTAs per SM
template <class P, class R>
struct HsSplitA {
  static constexpr int NT = 128, EV = 4, CTAS = 3;
  static constexpr size_t o_proptab = 0;
  static constexpr size_t o_md = align_up(o_proptab + 8 * P::NPROP, 16);
  static constexpr size_t o_mconst = align_up(o_md + 16 * P::NMOM, 16);
  static constexpr size_t o_p = align_up(o_mconst + 32, 16);
  static constexpr size_t o_K = align_up(o_p + 8 * EV * P::NPAR * 4, 16);
  static constexpr size_t o_pr = align_up(o_K + sizeof(R) * EV * P::NMOM * 4, 16);
  static constexpr size_t o_cur = align_up(o_pr + 2 * sizeof(R) * EV * P::NPROP, 16);
  static constexpr size_t bytes = o_cur + sizeof(W4<R>) * EV * P::HS_NSLOT;
  static_assert(bytes <= 232448, "shared memory per CTA above the 227 KB limit");
};

template <class P, class R>
__global__ void __launch_bounds__(HsSplitA<P, R>::NT, HsSplitA<P, R>::CTAS)
    sigmakin_hs_currents_kernel(SigArgs a, Couplings<R> cp, int64_t first, int64_t last, uint4* __restrict__ rec) {
  using L = HsSplitA<P, R>;
  using RC = HsRecord<P, R>;
  constexpr int NT = L::NT;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x;
  const int64_t e0 = first + (int64_t)blockIdx.x * L::EV;
  if (e0 >= last) return;
  const int nev = (int)min((int64_t)L::EV, last - e0);
  uint4* curs = reinterpret_cast<uint4*>(smem + L::o_cur);
  hs_setup_words<P, R, L>(smem, a.pp);
  hs_load_momenta<P, R, L>(smem, a.mom, a.nevt, e0, nev);
  __syncthreads();
  const HsGroup cta{0, NT, tid, 0, nev, 0};
  hs_tables<P, R, L>(smem, a.pp, cta, curs, cp);
  const R* Kall = reinterpret_cast<const R*>(smem + L::o_K);
  const cx<R>* prall = reinterpret_cast<const cx<R>*>(smem + L::o_pr);
  const HsItem* items = P::hs_items();
#pragma unroll
  for (int l = 1; l < P::HS_NLEVEL; ++l) {
    const int i0 = P::hs_level(l), ni = P::hs_level(l + 1) - i0, n = ni * nev;
    for (int t = tid; t < n; t += NT) {
      const int e = t / ni;
      const HsItem it = items[i0 + t - e * ni];
      hs_item<P, R>(it, Slots<R, P::HS_NSLOT>{curs + e * RC::CUR}, Kall + e * P::NMOM * 4, prall + e * P::NPROP,
                    cp);
    }
    __syncthreads();
  }
  const uint4* ks = reinterpret_cast<const uint4*>(smem + L::o_K);
  uint4* out = rec + (e0 - first) * RC::WORDS;
  for (int t = tid; t < nev * RC::WORDS; t += NT) {
    const int e = t / RC::WORDS, w = t - e * RC::WORDS;
    out[t] = w < RC::CUR ? curs[e * RC::CUR + w] : ks[e * RC::KW + (w - RC::CUR)];
  }
}

template <class P, class R>
__global__ void __launch_bounds__(HsCfg<P, R>::NT, HsCfg<P, R>::CTAS)
    sigmakin_hs_amplitudes_kernel(SigArgs a, Couplings<R> cp, int64_t first, int64_t last, const uint4* __restrict__ rec) {
  hs_sigmakin_body<P, R, CS_SIMT, kSrcRecords>(a, cp, first, last, rec);
}

template <class P, class R>
struct SplitLaunch {
  static cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(sigmakin_hs_currents_kernel<P, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HsSplitA<P, R>::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sigmakin_hs_amplitudes_kernel<P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)HsLayout<P, R, CS_SIMT>::bytes);
  }
  static cudaError_t currents(const SigArgs& a, const Couplings<R>& cp, int64_t first, int64_t last, uint4* rec,
                              cudaStream_t s) {
    using L = HsSplitA<P, R>;
    const int64_t grid = (last - first + L::EV - 1) / L::EV;
    sigmakin_hs_currents_kernel<P, R><<<(unsigned)grid, L::NT, L::bytes, s>>>(a, cp, first, last, rec);
    return cudaGetLastError();
  }
  static cudaError_t amplitudes(const SigArgs& a, const Couplings<R>& cp, int64_t first, int64_t last,
                                const uint4* rec, cudaStream_t s) {
    using C = HsCfg<P, R>;
    const int64_t grid = (last - first + C::EVMIN - 1) / C::EVMIN;
    sigmakin_hs_amplitudes_kernel<P, R>
        <<<(unsigned)grid, C::NT, HsLayout<P, R, CS_SIMT>::bytes, s>>>(a, cp, first, last, rec);
    return cudaGetLastError();
  }
};

}  // namespace mg

namespace mg {

// One batch through the split kernels: chunk = workspace / (2 records), a
// multiple of the currents kernel's events per CTA; the graph key holds every
// launch argument, so a call with other buffers or parameters re-captures.
template <class P, class R>
cudaError_t launch_split_impl(int proc, const SigLaunch& l, const Couplings<R>& cp, int mode, void* ws,
                              int64_t ws_bytes, cudaStream_t s) {
  using RC = HsRecord<P, R>;
  constexpr int64_t rec_bytes = (int64_t)RC::WORDS * 16;
  int64_t chunk = ws_bytes / (2 * rec_bytes);
  // whole waves of the amplitudes kernel (all helicities good) where the
  // workspace allows: a partial last wave per chunk idles SMs
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaGetLastError();
  const int64_t wave = (int64_t)nsm * HsCfg<P, R>::CTAS * HsCfg<P, R>::EVMIN;
  chunk -= chunk >= wave ? chunk % wave : chunk % HsSplitA<P, R>::EV;
  if (chunk < HsSplitA<P, R>::EV) return cudaErrorInvalidValue;
  if (l.nevt == 0) return cudaSuccess;
  if (chunk > l.nevt) chunk = (l.nevt + HsSplitA<P, R>::EV - 1) / HsSplitA<P, R>::EV * HsSplitA<P, R>::EV;
  struct Key {
    int proc_mode;
    int device;  // a graph belongs to the device it was captured on
    SigArgs a;
    Couplings<R> cp;
    void* ws;
    int64_t chunk;
  } key;
  std::memset(&key, 0, sizeof key);  // padding compared too
  key.proc_mode = proc * 16 + mode;
  key.device = dev;
  key.a = SigArgs{l.nevt, l.mom, l.mask, l.me, nullptr, l.pp, l.hel_rnd, l.hel_out, l.col_rnd, l.col_out};
  key.cp = cp;
  key.ws = ws;
  key.chunk = chunk;
  const SigArgs a = key.a;
  SplitOps ops;
  ops.prepare = [] { return SplitLaunch<P, R>::prepare(); };
  ops.currents = [a, cp](int64_t f, int64_t e, void* rec, cudaStream_t st) {
    return SplitLaunch<P, R>::currents(a, cp, f, e, static_cast<uint4*>(rec), st);
  };
  ops.amplitudes = [a, cp](int64_t f, int64_t e, const void* rec, cudaStream_t st) {
    return SplitLaunch<P, R>::amplitudes(a, cp, f, e, static_cast<const uint4*>(rec), st);
  };
  char* b0 = static_cast<char*>(ws);
  return run_split_graph(&key, sizeof key, l.nevt, chunk, b0, b0 + chunk * rec_bytes, ops, s);
}

}  // namespace mg

// One translation unit per process and precision (they compile in parallel):
// MG_DEFINE_SPLIT_LAUNCHERS with the FP32 kernels and the dispatcher,
// MG_INSTANTIATE_SPLIT_FP64 with the FP64 kernels.
#define MG_DEFINE_SPLIT_LAUNCHERS(N)                                                                    \
  namespace mg {                                                                                         \
  extern template cudaError_t launch_split_impl<Proc##N, double>(int, const SigLaunch&,                 \
                                                                  const Couplings<double>&, int, void*, \
                                                                  int64_t, cudaStream_t);               \
  int64_t split_record_bytes_p##N(int mode) {                                                           \
    return mode == 0 ? (int64_t)HsRecord<Proc##N, double>::WORDS * 16                                    \
                     : (int64_t)HsRecord<Proc##N, float>::WORDS * 16;                                    \
  }                                                                                                      \
  cudaError_t launch_sigmakin_split_p##N(const SigLaunch& l, int mode, void* ws, int64_t ws_bytes,      \
                                         cudaStream_t s) {                                               \
    if (mode == 0) return launch_split_impl<Proc##N, double>(N, l, l.cd, mode, ws, ws_bytes, s);         \
    if (mode == 2) return launch_split_impl<Proc##N, float>(N, l, l.cf, mode, ws, ws_bytes, s);          \
    return cudaErrorInvalidValue;                                                                        \
  }                                                                                                      \
  }

#define MG_INSTANTIATE_SPLIT_FP64(N)                                                                    \
  namespace mg {                                                                                         \
  template cudaError_t launch_split_impl<Proc##N, double>(int, const SigLaunch&, const Couplings<double>&, \
                                                          int, void*, int64_t, cudaStream_t);           \
  }
