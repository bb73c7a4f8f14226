/*
 * mg.h -- C ABI of the GB300 matrix-element library (libmg.so).
 *
 * Per-event tree-level squared matrix elements for the data-parallel
 * workflow of arXiv:2106.12631 (Valassi, Roiser, Mattelaer, Hageboeck):
 * uniform random numbers -> RAMBO momenta and weights -> helicity filtering ->
 * |M|^2 from helicity amplitudes and the colour-flow colour sum -> event sum.
 *
 * Processes (proc ids):
 *   1  e+ e- -> mu+ mu-   (photon + Z, 2 diagrams, 16 helicities, 1 colour flow)
 *   2  g g -> t t~        (3 diagrams, 16 helicities, 2 colour flows)
 *   3  g g -> t t~ g      (16 diagrams, 32 helicities, 6 colour flows)
 *   4  g g -> t t~ g g    (123 diagrams, 64 helicities, 24 colour flows)
 *
 * Conventions shared by every entry point
 *  - Arrays are device pointers unless the name starts with h_; they are
 *    structure-of-arrays with the event index fastest (the paper's AOSOA
 *    layout, Sec. 4, with a single page spanning all events):
 *      rnd[k * nevt + i]                 random number k of event i
 *      mom[((p * 4) + mu) * nevt + i]    particle p, component mu = (E, px, py, pz)
 *      me[i], wgt[i]                     per-event outputs
 *    Particle order is the process string above; legs 0 and 1 are the beams.
 *  - Device pointers must be 16-byte aligned (MG_ERR_ALIGN otherwise).
 *  - The caller allocates and frees every buffer; the library keeps no
 *    per-call allocations and no device state besides compiled kernels.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL =
 *    legacy default stream).  The return value reports argument validation
 *    and launch errors only; faults inside a kernel surface at the next
 *    synchronisation.  Nothing aborts and nothing throws across the ABI.
 *  - nevt == 0 is valid and enqueues nothing (mg_event_sum writes zeros).
 */
#ifndef MG_H_
#define MG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_ABI_VERSION 4

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = -1,     /* bad size, null pointer, bad mode or out-of-range value */
  MG_ERR_PROC = -2,    /* unknown process id */
  MG_ERR_ALIGN = -3,   /* a device pointer is not 16-byte aligned */
  MG_ERR_CUDA = -5,    /* a CUDA call failed; see mg_last_cuda_error() */
  MG_ERR_SPACE = -6    /* workspace or scratch smaller than required */
} mg_status;

/* Precision modes of mg_sigmakin (the paper's build-time precision switch, Sec. 4,
 * extended to a mixed mode). */
typedef enum {
  MG_FP64 = 0,        /* everything in FP64 */
  MG_MIXED = 1,       /* FP32 wavefunctions, currents and amplitudes; FP64 momenta,
                         momentum sums, propagator invariants and helicity/event
                         sums; colour sum on CUDA cores in FP32 below 48 colour
                         flows, on the tensor cores from 48 flows on */
  MG_MIXED_SIMT = 2,  /* MG_MIXED with the colour sum on CUDA cores in FP32 */
  MG_FP64_UNROLLED = 3,   /* MG_FP64 with every helicity recomputing all its currents */
  MG_MIXED_UNROLLED = 4,  /* MG_MIXED_TC with every helicity recomputing all its currents */
  MG_MIXED_TC = 5     /* MG_MIXED with the colour sum on the tensor cores
                         (split-BF16 operands, FP32 accumulation) */
} mg_mode;
/* Modes 0-2 and 5 evaluate each off-shell current once per event for each
 * helicity combination of its own external legs, and each diagram as the
 * contraction of one of its currents with the amputated current of the others
 * (also shared across helicities); modes 3-4 run one unrolled program per
 * helicity (the organisation of the paper's SIGMAKIN).  Same results up to
 * rounding. */

typedef struct {
  int npar;          /* external particles */
  int nhel;          /* helicity combinations (2^npar) */
  int ncolor;        /* colour flows */
  int ndiagrams;     /* Feynman diagrams (a four-gluon vertex counts once) */
  int namplitudes;   /* amplitude terms (four-gluon vertices split in 3) */
  int nrand;         /* random numbers RAMBO consumes per event (4 per final particle) */
  double mass[8];    /* particle masses for the current parameters [GeV] */
} mg_process_info;

/* Standard-Model inputs.  Defaults: mz 91.188, wz 2.441, alpha_inv 132.507,
 * sw2 0.2222, mt 173, wt 1.491, alpha_s 0.118. */
typedef struct {
  double mz, wz;       /* Z mass and width [GeV] */
  double alpha_inv;    /* 1 / alpha_em */
  double sw2;          /* sin^2 theta_W */
  double mt, wt;       /* top mass and width [GeV] */
  double alpha_s;      /* strong coupling */
} mg_params;

/* Static description of a process.  Host only.  MG_ERR_PROC for a bad id. */
int mg_get_process_info(int proc, mg_process_info* out);

/* Replace the physics parameters used by subsequent launches (host state of
 * the library, read at launch time; not thread safe against concurrent
 * launches).  MG_ERR_ARG for non-finite or non-physical values. */
int mg_set_params(const mg_params* p);
int mg_get_params(mg_params* out);

/* RAMBO (Sec. 3, "RAMBO" step of the toy workflow; Kleiss, Stirling, Ellis).
 * rnd: [nrows][nevt] uniforms in (0,1); rows 4i..4i+3 drive final particle i
 * (cos theta = 2 r1 - 1, phi = 2 pi r2, E ~ -log(r3 r4)); rows beyond
 * 4*nfinal are ignored.  Output mom [npar][4][nevt] (beams along +z and -z at
 * ecm/2 each) and wgt [nevt], the flat phase-space volume element without
 * (2 pi) factors.  FP64.  MG_ERR_ARG if nrows < 4*nfinal or the final masses
 * exceed ecm. */
int mg_rambo(int proc, int64_t nevt, double ecm, const double* rnd, int nrows,
             double* mom, double* wgt, void* stream);

/* Helicity filtering (Sec. 2: allowed helicity combinations are found on a
 * small set of events).  Computes |M_h|^2 in FP64 for every helicity h on the
 * nevt events of mom and sets mask[h] = 1 if any event gives a non-zero
 * value, else 0.  mask: [nhel] int32, overwritten (zeroed on the stream first).
 * Typical nevt: 16. */
int mg_filter_helicities(int proc, int64_t nevt, const double* mom, int32_t* mask, void* stream);

/* Squared matrix elements (the paper's SIGMAKIN, Sec. 4): for every event,
 *   me = 1/(helicity avg x colour avg x identical-particle factor)
 *        x sum_{h : mask[h] != 0} J_h^dagger C J_h
 * with J_h the colour-flow dual amplitudes of helicity h (Sec. 2) and C the
 * colour matrix.  mask: [nhel] int32 from mg_filter_helicities (an all-zero
 * mask gives me = 0).  mode: mg_mode.  me has units GeV^(8 - 2 npar):
 * dimensionless for 2 -> 2, GeV^-2 for 2 -> 3, GeV^-4 for 2 -> 4. */
int mg_sigmakin(int proc, int64_t nevt, const double* mom, const int32_t* mask, double* me, int mode,
                void* stream);

/* Gradient of the matrix element with respect to the random numbers (not in
 * the paper): for every event i, grad[k][i] = gout[i] * d me_i / d rnd[k][i],
 * through RAMBO and the helicity amplitudes by a hand-written adjoint (the
 * diagram program of each helicity is recomputed, then reversed; RAMBO's
 * Newton step enters through its implicit-function derivative).  rnd: [nrows]
 * [nevt] as for mg_rambo; rows beyond 4*nfinal get exactly 0.  gout: [nevt]
 * dL/dme or NULL for 1.  me: [nevt] receives the matrix elements (or NULL).
 * mode: MG_FP64 (FP64 forward and adjoint) or MG_MIXED / MG_MIXED_SIMT /
 * MG_MIXED_TC (FP32 forward and adjoint on CUDA cores; FP64 RAMBO, propagator
 * denominators and sums).
 * Available for proc 2 (g g -> t t~) and 3 (g g -> t t~ g); MG_ERR_PROC
 * otherwise. */
int mg_sigmakin_grad(int proc, int64_t nevt, double ecm, const double* rnd, int nrows, const int32_t* mask,
                     const double* gout, double* grad, double* me, int mode, void* stream);

/* Event accumulation in FP64 (Sec. 3: average matrix element of a run):
 * out3 = (sum_i wgt_i me_i, sum_i (wgt_i me_i)^2, nevt), by a two-pass tree
 * reduction whose order depends only on nevt (bitwise reproducible).
 * scratch: device buffer of at least mg_event_sum_scratch_bytes(nevt) bytes,
 * owned by the caller, overwritten.  MG_ERR_SPACE if too small. */
int64_t mg_event_sum_scratch_bytes(int64_t nevt);
int mg_event_sum(int64_t nevt, const double* me, const double* wgt, double* out3, void* scratch,
                 int64_t scratch_bytes, void* stream);

/* The event sum above without caller scratch, for callers that cannot
 * allocate device memory: code that runs while a stream is being captured into
 * a CUDA graph (cudaMalloc is not allowed there), host programs whose device
 * memory is owned by another framework's pool, or integrator loops that must
 * not trigger the device-wide synchronisation a cudaMalloc/cudaFree can cause.
 * The paper has no counterpart; this is a convenience of this library.
 * The partial sums live in a fixed array compiled into libmg.so, on every
 * device that loads the library, kept until the process exits: room for
 * mg_event_sum_noalloc_max_events() = 2^26 events (256 KiB per device).
 * Larger nevt returns MG_ERR_SPACE and launches nothing.  The call allocates
 * nothing.  Its first call on a device looks up that array's device address
 * (once per device, with the device current), so make the first call before
 * any stream capture.  That address is kept for the life of the device's
 * primary context: after cudaDeviceReset, or with another context made
 * current on the same device, it is stale, so do not call this function
 * then.  All calls share the array: calls that overlap on the GPU (two
 * streams, two host threads) race and give wrong sums; serialise them.
 * Results are identical to mg_event_sum's. */
int64_t mg_event_sum_noalloc_max_events(void);
int mg_event_sum_noalloc(int64_t nevt, const double* me, const double* wgt, double* out3, void* stream);

/* RAMBO and SIGMAKIN in one kernel (Sec. 3: random numbers -> RAMBO -> matrix
 * elements), for callers that need only me and the phase-space weight: no
 * momentum buffer, no momentum round trip through HBM.  Each CTA runs RAMBO
 * for its next group of events, one lane per event, while it computes the
 * current group.  me and wgt equal, bit for bit, mg_rambo (or
 * mg_rambo_seeded) followed by mg_sigmakin with the same mask and mode.  On
 * GB300 it saves memory, not time: RAMBO's FP64 work on one lane per event
 * takes longer than a group's matrix elements, so the kernel waits for it
 * (gg -> t t~ g g, 2^20 events, mixed: 44.5 ms against 22.2 ms for the two
 * kernels).
 * mg_sigmakin_rambo: uniforms rnd [nrows][nevt] (device), as mg_rambo.
 * mg_sigmakin_seeded: uniforms drawn on the device, as mg_rambo_seeded
 * (seed, first_event >= 0, first_event + nevt <= 2^57).
 * mask: [nhel] from mg_filter_helicities; mode: MG_FP64, MG_MIXED,
 * MG_MIXED_SIMT or MG_MIXED_TC (the helicity-shared kernels; the per-helicity
 * modes give MG_ERR_ARG).  me, wgt: device [nevt]. */
int mg_sigmakin_rambo(int proc, int64_t nevt, double ecm, const double* rnd, int nrows, const int32_t* mask,
                      int mode, double* me, double* wgt, void* stream);
int mg_sigmakin_seeded(int proc, int64_t nevt, double ecm, uint64_t seed, int64_t first_event,
                       const int32_t* mask, int mode, double* me, double* wgt, void* stream);

/* RAMBO with the uniforms drawn on the device (Sec. 3's random numbers fused
 * into the phase-space kernel; no random-number buffer): the uniform of event
 * i, row k is SplitMix64 used as a counter-based generator,
 *   key = mix(seed), z = mix(key + (64 (first_event + i) + k + 1) * 0x9E3779B97F4A7C15),
 *   u = ((z >> 11) + 0.5) 2^-53,
 * mix = SplitMix64's finaliser (Steele, Lea, Flood, OOPSLA 2014); rows
 * 0 .. 4 nfinal - 1 feed RAMBO as in mg_rambo, whose results these equal for
 * the same uniforms.  mom, wgt: device, as for mg_rambo.  first_event >= 0 and
 * first_event + nevt <= 2^57, else MG_ERR_ARG. */
int mg_rambo_seeded(int proc, int64_t nevt, double ecm, uint64_t seed, int64_t first_event, double* mom,
                    double* wgt, void* stream);

/* Cross section from the event sums (Sec. 3: the average of the weighted
 * matrix elements of a run gives the cross section): sums3 = {sum w me,
 * sum (w me)^2, N} from mg_event_sum (device); xsec2 (device) receives
 * sigma = (hbar c)^2 (2 pi)^(4 - 3 nfinal) / (2 s) * (sum w me) / N  in pb and
 * its Monte Carlo error from the sample variance (0 for N <= 1).  The flux
 * 1/(2 s) is that of massless beams; w is mg_rambo's flat weight. */
int mg_cross_section(int proc, double ecm, const double* sums3, double* xsec2, void* stream);

/* Hit-or-miss unweighting (the toy workflow's unweighted events): with
 * x_i = wgt_i me_i and u_i the generator's uniform for (seed, first_event + i,
 * row 63), event i is kept iff u_i * max_j x_j < x_i.  The kept event indices
 * (0-based within this batch) are written to idx in increasing order and their
 * number to *count (device int64).  idx must hold nevt entries (the worst case).
 * scratch: device, >= mg_unweight_scratch_bytes(nevt) bytes, else MG_ERR_SPACE.
 * Deterministic: the same inputs give the same indices.  nevt <= 2^41. */
int64_t mg_unweight_scratch_bytes(int64_t nevt);
int mg_unweight(int64_t nevt, const double* me, const double* wgt, uint64_t seed, int64_t first_event,
                int64_t* idx, int64_t* count, void* scratch, int64_t scratch_bytes, void* stream);

/* Batched matrix elements for an external integrator (Sec. 5: the MadEvent
 * bridge, where an existing event generator hands over a set of phase-space
 * points it prepared and receives their matrix elements, its 4-momenta passed
 * in its own layout): momenta as an array of structures
 * mom_aos[nevt][npar][4] (device; E, px, py, pz of every particle in the
 * process's leg order, incoming legs first, as mg_rambo returns them but event
 * by event) -> me[nevt] as mg_sigmakin (mask from mg_filter_helicities, mode as
 * mg_sigmakin).  Optional choices (modes 0-2 and 5; NULL outputs skip them,
 * a non-NULL output needs its uniforms, device [nevt] in [0, 1)), made per
 * event in FP64 by inverse-CDF sampling: the first index, in order, whose
 * running sum of weights exceeds u * (sum of the weights):
 *   hel_out (int32 [nevt], from hel_rnd): a good helicity, weights |M_h|^2
 *     (colour summed) in helicity-index order;
 *   col_out (int32 [nevt], from col_rnd): a colour flow s, weights
 *     sum over the good helicities of |J_s|^2 (Sec. 2, colour-flow method:
 *     J_s the coefficient of the chain (T^{a_s1} ... T^{a_sk})_{i_top j_antitop},
 *     s the k! orderings of the gluon legs, in leg order, in lexicographic
 *     order; one flow without colour).
 * Both are -1 for an event with me = 0.  workspace: device, >=
 * mg_batch_workspace_bytes(proc, nevt) bytes (the structure-of-arrays copy),
 * else MG_ERR_SPACE. */
int64_t mg_batch_workspace_bytes(int proc, int64_t nevt);
int mg_matrix_elements_batch(int proc, int64_t nevt, const double* mom_aos, const int32_t* mask, int mode,
                             const double* hel_rnd, const double* col_rnd, double* me, int32_t* hel_out,
                             int32_t* col_out, void* workspace, int64_t workspace_bytes, void* stream);

/* Kernel-split variant of mg_sigmakin (Sec. 4, future work: the single large
 * SIGMAKIN kernel split into smaller kernels orchestrated with CUDA Graphs),
 * kept for comparison with the single kernel.  Same inputs and result as
 * mg_sigmakin (mom [npar][4][nevt], mask, me [nevt]; mode MG_FP64 = 0 or
 * MG_MIXED_SIMT = 2 only, else MG_ERR_ARG): the events go through in chunks;
 * for each chunk one kernel computes every current variant and writes them to
 * workspace, a second reads them back and computes amplitudes, colour and
 * helicity sums.  workspace: device, two chunk buffers; chunk = workspace /
 * (2 x per-event record), so at least 8 records (MG_ERR_SPACE otherwise);
 * mg_sigmakin_split_workspace_bytes returns the size whose two buffers
 * together hold at most 96 MiB (they stay in L2).  The launches of one call are
 * captured into a CUDA graph, instantiated once and replayed while the
 * arguments, buffers and parameters are unchanged (one cached graph per
 * library, calls serialised by a mutex). */
int64_t mg_sigmakin_split_workspace_bytes(int proc, int mode, int64_t nevt);
int mg_sigmakin_split(int proc, int64_t nevt, const double* mom, const int32_t* mask, int mode, double* me,
                      void* workspace, int64_t workspace_bytes, void* stream);

/* End-to-end pipeline from HOST buffers (copies inside): h_rnd [nrows][nevt]
 * -> host-to-device copy -> RAMBO -> SIGMAKIN (mask from mg_filter_helicities,
 * on the device) -> device-to-host copy of me (and wgt if h_wgt != NULL) and,
 * if h_sums != NULL, of the FP64 event sum {sum w me, sum (w me)^2, nevt} of
 * mg_event_sum (3 doubles).  Host buffers should be pinned for asynchronous
 * copies.  workspace: device buffer of at least
 * mg_pipeline_workspace_bytes(proc, nevt, nrows) bytes.  Enqueued on stream;
 * the host buffers are valid after the stream synchronises. */
int64_t mg_pipeline_workspace_bytes(int proc, int64_t nevt, int nrows);
int mg_pipeline_host(int proc, int64_t nevt, double ecm, const double* h_rnd, int nrows, const int32_t* mask,
                     int mode, double* h_me, double* h_wgt, double* h_sums, void* workspace,
                     int64_t workspace_bytes, void* stream);

/* Human-readable status; the CUDA error code of the last MG_ERR_CUDA. */
const char* mg_status_string(int status);
int mg_last_cuda_error(void);
int mg_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H_ */
