// C ABI (include/mg.h): argument validation, parameter state, dispatch.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mg.h"
#include "launch.h"
#include "process.cuh"
#include "rng.cuh"

namespace {

struct ProcDesc {
  int npar, nhel, ncolor, ndiagrams, namps;
  int top[8];  // 1 if the leg is a top quark
};
// counts cross-checked against the generated process headers at compile time below
const ProcDesc kProcs[5] = {
    {0, 0, 0, 0, 0, {0}},
    {4, 16, 1, 2, 2, {0, 0, 0, 0}},
    {4, 16, 2, 3, 3, {0, 0, 1, 1}},
    {5, 32, 6, 16, 18, {0, 0, 1, 1, 0}},
    {6, 64, 24, 123, 159, {0, 0, 1, 1, 0, 0}},
};

static_assert(mg::Proc1::NDIAGRAMS == 2 && mg::Proc1::NCOLOR == 1 && mg::Proc1::NAMPS == 2, "proc 1");
static_assert(mg::Proc2::NDIAGRAMS == 3 && mg::Proc2::NCOLOR == 2 && mg::Proc2::NAMPS == 3, "proc 2");
static_assert(mg::Proc3::NDIAGRAMS == 16 && mg::Proc3::NCOLOR == 6 && mg::Proc3::NAMPS == 18, "proc 3");
static_assert(mg::Proc4::NDIAGRAMS == 123 && mg::Proc4::NCOLOR == 24 && mg::Proc4::NAMPS == 159, "proc 4");

std::mutex g_mu;
mg_params g_params = {91.188, 2.441, 132.507, 0.2222, 173.0, 1.491, 0.118};
thread_local int g_last_cuda = 0;

bool valid_proc(int proc) { return proc >= 1 && proc <= 4; }
bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

mg_params params_snapshot() {
  std::lock_guard<std::mutex> g(g_mu);
  return g_params;
}

template <class R>
mg::Couplings<R> couplings(const mg_params& p) {
  const double e = std::sqrt(4.0 * M_PI / p.alpha_inv);
  const double gs = std::sqrt(4.0 * M_PI * p.alpha_s);
  mg::Couplings<R> c;
  c.gs = R(gs);
  c.gs2 = R(gs * gs);
  c.ee = R(e);
  c.gz = R(e / std::sqrt(p.sw2 * (1.0 - p.sw2)));
  c.gzl = R(-0.5 + p.sw2);
  c.gzr = R(p.sw2);
  c.mt = R(p.mt);
  return c;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MG_OK;
  g_last_cuda = (int)e;
  return MG_ERR_CUDA;
}

mg::SigLaunch sig_launch(int64_t nevt, const double* mom, const int32_t* mask, double* me, int32_t* mask_out) {
  const mg_params p = params_snapshot();
  mg::SigLaunch l;
  l.nevt = nevt;
  l.mom = mom;
  l.mask = mask;
  l.me = me;
  l.mask_out = mask_out;
  l.pp = mg::PhysParams{p.mz, p.wz, p.mt, p.wt};
  l.cd = couplings<double>(p);
  l.cf = couplings<float>(p);
  return l;
}

cudaError_t dispatch_sigmakin(int proc, const mg::SigLaunch& l, int mode, cudaStream_t s) {
  switch (proc) {
    case 1: return mg::launch_sigmakin_p1(l, mode, s);
    case 2: return mg::launch_sigmakin_p2(l, mode, s);
    case 3: return mg::launch_sigmakin_p3(l, mode, s);
    case 4: return mg::launch_sigmakin_p4(l, mode, s);
  }
  return cudaErrorInvalidValue;
}

int64_t split_record_bytes(int proc, int mode) {
  switch (proc) {
    case 1: return mg::split_record_bytes_p1(mode);
    case 2: return mg::split_record_bytes_p2(mode);
    case 3: return mg::split_record_bytes_p3(mode);
    default: return mg::split_record_bytes_p4(mode);
  }
}

cudaError_t dispatch_sigmakin_rambo(int proc, const mg::SigLaunch& l, int mode, cudaStream_t s) {
  switch (proc) {
    case 1: return mg::launch_sigmakin_rambo_p1(l, mode, s);
    case 2: return mg::launch_sigmakin_rambo_p2(l, mode, s);
    case 3: return mg::launch_sigmakin_rambo_p3(l, mode, s);
    case 4: return mg::launch_sigmakin_rambo_p4(l, mode, s);
  }
  return cudaErrorInvalidValue;
}

int rambo_setup(int proc, double ecm, mg::RamboSetup& st);

// mg_sigmakin_rambo (seeded = false: uniforms from rnd) and mg_sigmakin_seeded
int sigmakin_rambo(int proc, int64_t nevt, double ecm, const double* rnd, int nrows, bool seeded, uint64_t seed,
                   int64_t first_event, const int32_t* mask, int mode, double* me, double* wgt, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  const ProcDesc& d = kProcs[proc];
  if (nevt < 0 || !(ecm > 0) || !std::isfinite(ecm)) return MG_ERR_ARG;
  if (mode != MG_FP64 && mode != MG_MIXED && mode != MG_MIXED_SIMT && mode != MG_MIXED_TC) return MG_ERR_ARG;
  if (!seeded && nrows < 4 * (d.npar - 2)) return MG_ERR_ARG;
  if (seeded && (first_event < 0 || first_event > ((int64_t)1 << 57) - nevt)) return MG_ERR_ARG;
  mg::RamboSetup st;
  if (int r = rambo_setup(proc, ecm, st)) return r;
  if (nevt == 0) return MG_OK;
  if ((!seeded && !rnd) || !mask || !me || !wgt) return MG_ERR_ARG;
  if ((!seeded && !aligned(rnd)) || !aligned(mask) || !aligned(me) || !aligned(wgt)) return MG_ERR_ALIGN;
  if (nevt > (int64_t)INT32_MAX) return MG_ERR_ARG;
  mg::SigLaunch l = sig_launch(nevt, nullptr, mask, me, nullptr);
  l.rnd = seeded ? nullptr : rnd;
  l.wgt = wgt;
  l.ecm = ecm;
  l.key = seeded ? mg::sm64_mix(seed) : 0;
  l.first_event = seeded ? first_event : 0;
  l.st = st;
  return cuda_status(dispatch_sigmakin_rambo(proc, l, mode, (cudaStream_t)stream));
}

int rambo_setup(int proc, double ecm, mg::RamboSetup& st) {
  const ProcDesc& d = kProcs[proc];
  const mg_params p = params_snapshot();
  const int n = d.npar - 2;
  double f1 = 1.0, f2 = 1.0;
  for (int k = 2; k <= n - 1; ++k) f1 *= k;
  for (int k = 2; k <= n - 2; ++k) f2 *= k;
  st.w0 = std::pow(M_PI / 2.0, n - 1) * std::pow(ecm * ecm, n - 2) / (f1 * f2);
  double msum = 0.0;
  st.massive = 0;
  for (int i = 0; i < 4; ++i) st.m2[i] = 0.0;
  for (int i = 0; i < n; ++i) {
    const double m = d.top[2 + i] ? p.mt : 0.0;
    st.m2[i] = m * m;
    msum += m;
    if (m != 0.0) st.massive = 1;
  }
  if (!(msum < ecm)) return MG_ERR_ARG;
  st.xi0 = std::sqrt(1.0 - (msum / ecm) * (msum / ecm));
  return MG_OK;
}

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" {

int mg_abi_version(void) { return MG_ABI_VERSION; }
int mg_last_cuda_error(void) { return g_last_cuda; }

const char* mg_status_string(int s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_PROC: return "unknown process id";
    case MG_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_SPACE: return "workspace or scratch too small";
  }
  return "unknown status";
}

int mg_get_process_info(int proc, mg_process_info* out) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (!out) return MG_ERR_ARG;
  const ProcDesc& d = kProcs[proc];
  const mg_params p = params_snapshot();
  std::memset(out, 0, sizeof(*out));
  out->npar = d.npar;
  out->nhel = d.nhel;
  out->ncolor = d.ncolor;
  out->ndiagrams = d.ndiagrams;
  out->namplitudes = d.namps;
  out->nrand = 4 * (d.npar - 2);
  for (int i = 0; i < d.npar; ++i) out->mass[i] = d.top[i] ? p.mt : 0.0;
  return MG_OK;
}

int mg_set_params(const mg_params* p) {
  if (!p) return MG_ERR_ARG;
  const double v[7] = {p->mz, p->wz, p->alpha_inv, p->sw2, p->mt, p->wt, p->alpha_s};
  for (double x : v)
    if (!std::isfinite(x)) return MG_ERR_ARG;
  if (p->mz <= 0 || p->wz < 0 || p->alpha_inv <= 0 || p->sw2 <= 0 || p->sw2 >= 1 || p->mt < 0 || p->wt < 0 ||
      p->alpha_s <= 0)
    return MG_ERR_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  g_params = *p;
  return MG_OK;
}

int mg_get_params(mg_params* out) {
  if (!out) return MG_ERR_ARG;
  *out = params_snapshot();
  return MG_OK;
}

int mg_rambo(int proc, int64_t nevt, double ecm, const double* rnd, int nrows, double* mom, double* wgt,
             void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  const ProcDesc& d = kProcs[proc];
  if (nevt < 0 || !(ecm > 0) || !std::isfinite(ecm) || nrows < 4 * (d.npar - 2)) return MG_ERR_ARG;
  mg::RamboSetup st;
  if (int r = rambo_setup(proc, ecm, st)) return r;
  if (nevt == 0) return MG_OK;
  if (!rnd || !mom || !wgt) return MG_ERR_ARG;
  if (!aligned(rnd) || !aligned(mom) || !aligned(wgt)) return MG_ERR_ALIGN;
  if (nevt > (int64_t)INT32_MAX * 64) return MG_ERR_ARG;
  return cuda_status(mg::launch_rambo(d.npar - 2, nevt, ecm, rnd, mom, wgt, st, (cudaStream_t)stream));
}

int mg_rambo_seeded(int proc, int64_t nevt, double ecm, uint64_t seed, int64_t first_event, double* mom,
                    double* wgt, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  const ProcDesc& d = kProcs[proc];
  if (nevt < 0 || first_event < 0 || !(ecm > 0) || !std::isfinite(ecm)) return MG_ERR_ARG;
  if (first_event > ((int64_t)1 << 57) - nevt) return MG_ERR_ARG;  // event counters stay below 2^57
  mg::RamboSetup st;
  if (int r = rambo_setup(proc, ecm, st)) return r;
  if (nevt == 0) return MG_OK;
  if (!mom || !wgt) return MG_ERR_ARG;
  if (!aligned(mom) || !aligned(wgt)) return MG_ERR_ALIGN;
  if (nevt > (int64_t)INT32_MAX * 64) return MG_ERR_ARG;
  return cuda_status(
      mg::launch_rambo(d.npar - 2, nevt, ecm, nullptr, mom, wgt, st, (cudaStream_t)stream, seed, first_event));
}

int mg_sigmakin_rambo(int proc, int64_t nevt, double ecm, const double* rnd, int nrows, const int32_t* mask,
                      int mode, double* me, double* wgt, void* stream) {
  return sigmakin_rambo(proc, nevt, ecm, rnd, nrows, false, 0, 0, mask, mode, me, wgt, stream);
}

int mg_sigmakin_seeded(int proc, int64_t nevt, double ecm, uint64_t seed, int64_t first_event,
                       const int32_t* mask, int mode, double* me, double* wgt, void* stream) {
  return sigmakin_rambo(proc, nevt, ecm, nullptr, 0, true, seed, first_event, mask, mode, me, wgt, stream);
}

int mg_cross_section(int proc, double ecm, const double* sums3, double* xsec2, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (!(ecm > 0) || !std::isfinite(ecm) || !sums3 || !xsec2) return MG_ERR_ARG;
  if (!aligned(sums3) || !aligned(xsec2)) return MG_ERR_ALIGN;
  // sigma = (hbar c)^2 (2 pi)^(4 - 3 n) / (2 s) * mean(w |M|^2); (hbar c)^2 = 0.3893793721 mb GeV^2
  const int nf = kProcs[proc].npar - 2;
  const double hbarc2_pb = 0.3893793721e9;
  const double norm = hbarc2_pb * std::pow(2.0 * M_PI, 4.0 - 3.0 * nf) / (2.0 * ecm * ecm);
  return cuda_status(mg::launch_cross_section(sums3, norm, xsec2, (cudaStream_t)stream));
}

int64_t mg_unweight_scratch_bytes(int64_t nevt) {
  if (nevt < 0) return -1;
  return 8 * (1 + 2 * mg::unweight_blocks(nevt));
}

int mg_unweight(int64_t nevt, const double* me, const double* wgt, uint64_t seed, int64_t first_event,
                int64_t* idx, int64_t* count, void* scratch, int64_t scratch_bytes, void* stream) {
  if (nevt < 0 || first_event < 0 || !count) return MG_ERR_ARG;
  if (first_event > ((int64_t)1 << 57) - nevt) return MG_ERR_ARG;
  if (!aligned(count) || (me && !aligned(me)) || (wgt && !aligned(wgt)) || (idx && !aligned(idx)) ||
      (scratch && !aligned(scratch)))
    return MG_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (nevt == 0) return cuda_status(cudaMemsetAsync(count, 0, sizeof(int64_t), s));
  if (!me || !wgt || !idx || !scratch) return MG_ERR_ARG;
  if (nevt > (int64_t)INT32_MAX * 1024) return MG_ERR_ARG;
  if (scratch_bytes < mg_unweight_scratch_bytes(nevt)) return MG_ERR_SPACE;
  return cuda_status(mg::launch_unweight(nevt, me, wgt, seed, first_event, idx, count, (double*)scratch, s));
}

int64_t mg_batch_workspace_bytes(int proc, int64_t nevt) {
  if (!valid_proc(proc) || nevt < 0) return -1;
  return align256(8 * nevt * 4 * kProcs[proc].npar);
}

int mg_matrix_elements_batch(int proc, int64_t nevt, const double* mom_aos, const int32_t* mask, int mode,
                             const double* hel_rnd, const double* col_rnd, double* me, int32_t* hel_out,
                             int32_t* col_out, void* workspace, int64_t workspace_bytes, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (nevt < 0 || mode < 0 || mode > 5) return MG_ERR_ARG;
  if ((hel_out || col_out) && (mode == 3 || mode == 4)) return MG_ERR_ARG;  // choices: helicity-shared modes
  if ((hel_out && !hel_rnd) || (col_out && !col_rnd)) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!mom_aos || !mask || !me || !workspace) return MG_ERR_ARG;
  if (!aligned(mom_aos) || !aligned(mask) || !aligned(me) || !aligned(workspace) || (hel_out && !aligned(hel_out)) ||
      (col_out && !aligned(col_out)) || (hel_out && !aligned(hel_rnd)) || (col_out && !aligned(col_rnd)))
    return MG_ERR_ALIGN;
  if (workspace_bytes < mg_batch_workspace_bytes(proc, nevt)) return MG_ERR_SPACE;
  if (nevt > (int64_t)INT32_MAX * 16) return MG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double* soa = (double*)workspace;
  if (int r = cuda_status(mg::launch_aos_to_soa(nevt, kProcs[proc].npar, mom_aos, soa, s))) return r;
  mg::SigLaunch l = sig_launch(nevt, soa, mask, me, nullptr);
  l.hel_rnd = hel_out ? hel_rnd : nullptr;
  l.hel_out = hel_out;
  l.col_rnd = col_out ? col_rnd : nullptr;
  l.col_out = col_out;
  return cuda_status(dispatch_sigmakin(proc, l, mode, s));
}

int64_t mg_sigmakin_split_workspace_bytes(int proc, int mode, int64_t nevt) {
  if (!valid_proc(proc) || nevt < 0 || (mode != 0 && mode != 2)) return -1;
  const int64_t rec = split_record_bytes(proc, mode);
  // two chunk buffers of together at most 96 MiB (they stay in L2), 4 events at least
  int64_t chunk = ((int64_t)48 << 20) / rec;
  chunk -= chunk % 4;
  if (chunk < 4) chunk = 4;
  const int64_t need = (nevt + 3) / 4 * 4;
  return 2 * (need < chunk ? need : chunk) * rec;
}

int mg_sigmakin_split(int proc, int64_t nevt, const double* mom, const int32_t* mask, int mode, double* me,
                      void* workspace, int64_t workspace_bytes, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (nevt < 0 || (mode != 0 && mode != 2)) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!mom || !mask || !me || !workspace) return MG_ERR_ARG;
  if (!aligned(mom) || !aligned(mask) || !aligned(me) || !aligned(workspace)) return MG_ERR_ALIGN;
  if (workspace_bytes < 8 * split_record_bytes(proc, mode)) return MG_ERR_SPACE;
  if (nevt > (int64_t)INT32_MAX * 16) return MG_ERR_ARG;
  mg::SigLaunch l = sig_launch(nevt, mom, mask, me, nullptr);
  cudaStream_t s = (cudaStream_t)stream;
  switch (proc) {
    case 1: return cuda_status(mg::launch_sigmakin_split_p1(l, mode, workspace, workspace_bytes, s));
    case 2: return cuda_status(mg::launch_sigmakin_split_p2(l, mode, workspace, workspace_bytes, s));
    case 3: return cuda_status(mg::launch_sigmakin_split_p3(l, mode, workspace, workspace_bytes, s));
    default: return cuda_status(mg::launch_sigmakin_split_p4(l, mode, workspace, workspace_bytes, s));
  }
}

int mg_filter_helicities(int proc, int64_t nevt, const double* mom, int32_t* mask, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (nevt < 0) return MG_ERR_ARG;
  if (!mask) return MG_ERR_ARG;
  if (nevt > 0 && !mom) return MG_ERR_ARG;
  if (!aligned(mask) || (mom && !aligned(mom))) return MG_ERR_ALIGN;
  if (nevt > (1 << 20)) return MG_ERR_ARG;  // a filtering pass runs on a small event set
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = cuda_status(cudaMemsetAsync(mask, 0, sizeof(int32_t) * kProcs[proc].nhel, s))) return r;
  if (nevt == 0) return MG_OK;
  const mg::SigLaunch l = sig_launch(nevt, mom, nullptr, nullptr, mask);
  switch (proc) {
    case 1: return cuda_status(mg::launch_filter_p1(l, s));
    case 2: return cuda_status(mg::launch_filter_p2(l, s));
    case 3: return cuda_status(mg::launch_filter_p3(l, s));
    case 4: return cuda_status(mg::launch_filter_p4(l, s));
  }
  return MG_ERR_PROC;
}

int mg_sigmakin(int proc, int64_t nevt, const double* mom, const int32_t* mask, double* me, int mode,
                void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (nevt < 0 || mode < 0 || mode > 5) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!mom || !mask || !me) return MG_ERR_ARG;
  if (!aligned(mom) || !aligned(mask) || !aligned(me)) return MG_ERR_ALIGN;
  if (nevt > (int64_t)INT32_MAX) return MG_ERR_ARG;
  const mg::SigLaunch l = sig_launch(nevt, mom, mask, me, nullptr);
  return cuda_status(dispatch_sigmakin(proc, l, mode, (cudaStream_t)stream));
}

int mg_sigmakin_grad(int proc, int64_t nevt, double ecm, const double* rnd, int nrows, const int32_t* mask,
                     const double* gout, double* grad, double* me, int mode, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (proc != 2 && proc != 3) return MG_ERR_PROC;
  const ProcDesc& d = kProcs[proc];
  if (nevt < 0 || mode < 0 || mode > 5 || !(ecm > 0) || !std::isfinite(ecm) || nrows < 4 * (d.npar - 2))
    return MG_ERR_ARG;
  mg::RamboSetup st;
  if (int r = rambo_setup(proc, ecm, st)) return r;
  if (nevt == 0) return MG_OK;
  if (!rnd || !mask || !grad) return MG_ERR_ARG;
  if (!aligned(rnd) || !aligned(mask) || !aligned(grad) || (gout && !aligned(gout)) || (me && !aligned(me)))
    return MG_ERR_ALIGN;
  if (nevt > (int64_t)INT32_MAX) return MG_ERR_ARG;
  const mg_params p = params_snapshot();
  mg::GradLaunch l;
  l.nevt = nevt;
  l.ecm = ecm;
  l.rnd = rnd;
  l.nrows = nrows;
  l.mask = mask;
  l.gout = gout;
  l.grad = grad;
  l.me = me;
  l.pp = mg::PhysParams{p.mz, p.wz, p.mt, p.wt};
  l.cd = couplings<double>(p);
  l.cf = couplings<float>(p);
  l.st = st;
  cudaStream_t s = (cudaStream_t)stream;
  return cuda_status(proc == 2 ? mg::launch_grad_p2(l, mode, s) : mg::launch_grad_p3(l, mode, s));
}

int64_t mg_event_sum_scratch_bytes(int64_t nevt) {
  if (nevt < 0) return -1;
  return 16 * mg::event_sum_blocks(nevt) + 16;
}

int mg_event_sum(int64_t nevt, const double* me, const double* wgt, double* out3, void* scratch,
                 int64_t scratch_bytes, void* stream) {
  if (nevt < 0 || !out3) return MG_ERR_ARG;
  if (nevt > 0 && (!me || !wgt || !scratch)) return MG_ERR_ARG;
  if (!aligned(out3) || (me && !aligned(me)) || (wgt && !aligned(wgt)) || (scratch && !aligned(scratch)))
    return MG_ERR_ALIGN;
  if (scratch_bytes < mg_event_sum_scratch_bytes(nevt) && nevt > 0) return MG_ERR_SPACE;
  return cuda_status(mg::launch_event_sum(nevt, me, wgt, out3, (double*)scratch, (cudaStream_t)stream));
}

int64_t mg_event_sum_noalloc_max_events(void) { return mg::event_sum_noalloc_max_events(); }

int mg_event_sum_noalloc(int64_t nevt, const double* me, const double* wgt, double* out3, void* stream) {
  if (nevt < 0 || !out3) return MG_ERR_ARG;
  if (nevt > mg::event_sum_noalloc_max_events()) return MG_ERR_SPACE;
  if (nevt > 0 && (!me || !wgt)) return MG_ERR_ARG;
  if (!aligned(out3) || (me && !aligned(me)) || (wgt && !aligned(wgt))) return MG_ERR_ALIGN;
  return cuda_status(mg::launch_event_sum_noalloc(nevt, me, wgt, out3, (cudaStream_t)stream));
}

int64_t mg_pipeline_workspace_bytes(int proc, int64_t nevt, int nrows) {
  if (!valid_proc(proc) || nevt < 0 || nrows < 0) return -1;
  const int64_t n = nevt;
  return align256(8 * n * nrows) + align256(8 * n * 4 * kProcs[proc].npar) + 2 * align256(8 * n) + align256(8 * 3) +
         align256(mg_event_sum_scratch_bytes(n));
}

int mg_pipeline_host(int proc, int64_t nevt, double ecm, const double* h_rnd, int nrows, const int32_t* mask,
                     int mode, double* h_me, double* h_wgt, double* h_sums, void* workspace,
                     int64_t workspace_bytes, void* stream) {
  if (!valid_proc(proc)) return MG_ERR_PROC;
  if (nevt < 0 || mode < 0 || mode > 5 || nrows < 4 * (kProcs[proc].npar - 2)) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!h_rnd || !mask || !h_me || !workspace) return MG_ERR_ARG;
  if (workspace_bytes < mg_pipeline_workspace_bytes(proc, nevt, nrows)) return MG_ERR_SPACE;
  if (!aligned(workspace) || !aligned(mask)) return MG_ERR_ALIGN;
  char* ws = (char*)workspace;
  double* d_rnd = (double*)ws;
  ws += align256(8 * nevt * nrows);
  double* d_mom = (double*)ws;
  ws += align256(8 * nevt * 4 * kProcs[proc].npar);
  double* d_wgt = (double*)ws;
  ws += align256(8 * nevt);
  double* d_me = (double*)ws;
  ws += align256(8 * nevt);
  double* d_sums = (double*)ws;
  ws += align256(8 * 3);
  double* d_scratch = (double*)ws;
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = cuda_status(cudaMemcpyAsync(d_rnd, h_rnd, 8 * nevt * nrows, cudaMemcpyHostToDevice, s))) return r;
  if (int r = mg_rambo(proc, nevt, ecm, d_rnd, nrows, d_mom, d_wgt, stream)) return r;
  if (int r = mg_sigmakin(proc, nevt, d_mom, mask, d_me, mode, stream)) return r;
  if (int r = cuda_status(cudaMemcpyAsync(h_me, d_me, 8 * nevt, cudaMemcpyDeviceToHost, s))) return r;
  if (h_wgt)
    if (int r = cuda_status(cudaMemcpyAsync(h_wgt, d_wgt, 8 * nevt, cudaMemcpyDeviceToHost, s))) return r;
  if (h_sums) {
    if (int r = mg_event_sum(nevt, d_me, d_wgt, d_sums, d_scratch, mg_event_sum_scratch_bytes(nevt), stream))
      return r;
    if (int r = cuda_status(cudaMemcpyAsync(h_sums, d_sums, 8 * 3, cudaMemcpyDeviceToHost, s))) return r;
  }
  return MG_OK;
}

}  // extern "C"
