/*
 * kbe.h -- C ABI of libkbe, a GB300 (sm_103a) implementation of the
 * Kadanoff-Baym time step of arXiv 2505.19467 ("GPU Acceleration of
 * Non-equilibrium Green's Function Calculation using OpenACC and CUDA
 * FORTRAN"), on one GPU.
 *
 * Problem (Sec. 2): lattice fermions with N_b bands on a 1-D ring or 2-D
 * L0 x L1 mesh (n_k = L0 L1 points k = 2 pi m / L), bare Bloch Hamiltonian
 * h0(k) from hopping matrices t(R), an on-site inter-band density-density
 * interaction U(t) v_ab (Eq. 2; v = 1 - delta is the paper's pair of bands),
 * and a Peierls drive h0(k - A(t) d). The library advances the lesser and
 * greater two-time Green's functions G^<, G^>(k; t_n, t_j) row by row
 * (Algorithm 1) with
 *   (a1) the second-Born self-energy on the new row (Eq. 7, k - q
 *        convolution),
 *   (a2) the collision integrals over the stored history (Eq. 6, trapezoid
 *        weights),
 *   (a3) the mean-field Hamiltonian and the step propagators,
 *   (a4) the predictor-corrector update of the row and the time diagonal,
 *   (a5) equal-time observables.
 *
 * Conventions for every entry point:
 *  - Complex numbers are interleaved (re, im) doubles ("c128").
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership. Host output arrays are caller-owned and must hold the
 *    documented number of elements.
 *  - Device pointers ("dev") are caller-owned device memory on the current
 *    CUDA device; work is enqueued on the given stream (NULL = legacy default
 *    stream) and the call returns before it completes.
 *  - A handle owns all device memory it allocates. Handles are not thread
 *    safe. All work of a handle is ordered on the stream given at creation.
 *  - Errors: a negative kbe_status; kbe_last_error() has the message. Device
 *    faults and non-finite results are sticky: the handle refuses further
 *    steps until kbe_reset().
 */
#ifndef KBE_H
#define KBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KBE_OK = 0,
  KBE_ERR_ARG = -1,         /* invalid argument (size, pointer, range)          */
  KBE_ERR_OOM = -2,         /* device allocation failed                         */
  KBE_ERR_CUDA = -3,        /* a CUDA call failed                               */
  KBE_ERR_STATE = -4,       /* call not valid in the handle's state             */
  KBE_ERR_NONFINITE = -5,   /* a NaN/Inf appeared in the propagated state       */
  KBE_ERR_TIMEOUT = -6,     /* a bounded device wait expired                    */
  KBE_ERR_UNSUPPORTED = -7, /* configuration not compiled in (e.g. N_b)         */
  KBE_ERR_INTERNAL = -8
} kbe_status;

/* Storage of the two-time history and arithmetic of the collision-integral
 * sweep (the dominant kernel). Everything else (self-energy, propagators,
 * the update of the newest rows, the time diagonal, observables) is FP64 in
 * every mode; the two newest rows are always kept in FP64. The history keeps
 * G^< and dG = G^< - G^> per block.
 *   FP64: history complex128, sweep in FP64 (DFMA).
 *   DF64: history as pairs of FP32 (hi, lo) per real part (the same 8 bytes;
 *         48-bit significand), sweep in double-float arithmetic on the FP32
 *         pipe: exact products (FMA) and error-free sums, FP64-level result.
 *   C64:  history complex64 (half the bytes), sweep in FP32: plain sums
 *         over groups of at most 32 products per output, the groups added
 *         into a compensated (error-free TwoSum) sum over the memory time.
 *   F16X2: history as split FP16 pairs, hi = fp16(S x), lo = fp16(S x - hi)
 *         per real part with S = 4096 (the same 8 bytes per complex number
 *         as C64; 22-bit significand, absolute error below 2^-37 for tiny
 *         entries), stored k-outer in the operand layout of the tensor cores;
 *         the sweep runs on the tensor cores (tcgen05.mma, FP16 products of
 *         the hi and lo parts, FP32 accumulation in tensor memory) with the
 *         coefficient rows split the same way under a power-of-two scale.
 *         N_b in {4, 8}. The self-energy is computed in complex FP32 as for
 *         C64; everything else is FP64. */
enum {
  KBE_PREC_FP64 = 0,
  KBE_PREC_DF64 = 1,
  KBE_PREC_C64 = 2,
  KBE_PREC_F16X2 = 3
};

typedef struct kbe_config {
  int nb;          /* bands N_b, one of 1,2,3,4,6,8,12,16                        */
  int dim;         /* 1 (ring, L[1] must be 1) or 2                              */
  int L[2];        /* mesh extents, n_k = L[0] * L[1] <= 4096                    */
  int nt_max;      /* rows t_0 .. t_{nt_max} are stored, 1 <= nt_max <= 65534    */
  double dt;       /* time step (> 0)                                            */
  double beta, mu; /* Fermi initial state f(h0(k)) at inverse temperature beta  */
  int precision;   /* KBE_PREC_*                                                 */
  int n_corr;      /* corrector passes of Algorithm 1 (its "max", >= 0)          */
  int hf;          /* 1: Hartree-Fock mean field in h                            */
  int paper_shift; /* 1: the -U(t) n_c one-body term of Eq. 2 on band N_b - 1    */
  double corr_tol; /* Algorithm 1's epsilon: > 0 stops the correctors of a step   *
                    * once max_{j,k,a,b} |G^<(t_n,t_j) - previous pass| <=        *
                    * corr_tol (decided on the device, no host round trip);       *
                    * 0: always n_corr passes                                     */
  int quadrature;  /* memory-integral weights of Eq. 6: KBE_QUAD_TRAPEZOID (the     *
                    * paper's second-order rule) or KBE_QUAD_GREGORY                */
} kbe_config;

/* Quadrature of the collision integrals over [0, t_m] (Eq. 6). Gregory: the
 * fourth-order rule with end weights 3/8, 7/6, 23/24 (in units of dt) at both
 * ends for m >= 5, and for m <= 4 the closed Newton-Cotes rule of the whole
 * interval (trapezoid, Simpson, Simpson 3/8, Boole). */
enum {
  KBE_QUAD_TRAPEZOID = 0,
  KBE_QUAD_GREGORY = 1
};

typedef struct kbe_handle kbe_handle;

/* Per-handle timing of the collision-integral sweep kernel (CUDA events on the
 * handle's stream), accumulated while profiling is enabled. */
typedef struct kbe_profile_stats {
  int sweep_launches;       /* sweep launches timed                               */
  double sweep_ms;          /* summed event time of those launches                */
  double sweep_flops;       /* algorithmic flops of those launches (24 n^2 N_b^3 n_k) */
  double sweep_flops_executed; /* flops the kernel executes (~16 n^2 N_b^3 n_k; FP64 at
                               * N_b <= 8: its FP64-pipe operations, ~(12 + 4/N_b)
                               * n^2 N_b^3 n_k, three-multiplication products) */
  double sweep_bytes;       /* algorithmic bytes (stored history read once + I row) */
  int launches;             /* all kernels launched while enabled                 */
  /* kbe_backward while enabled (CUDA events around each phase): the steps'
   * recomputation, the collision-row transposes, the Sigma-row transposes,
   * and the update / h transposes, in ms; and the flops of the collision-row
   * transposes (algorithmic count, 8 per complex multiply-add). */
  double backward_ms[4];
  double backward_sweep_flops;
} kbe_profile_stats;

/* ---------------------------------------------------------------------- */
/* handle API (Algorithm 1 on a resident two-time history)                 */
/* ---------------------------------------------------------------------- */

/* Create a handle. cfg is copied. stream is a cudaStream_t (NULL: default).
 * Allocates the lower-triangle history (nt_max+1)(nt_max+2)/2 blocks of
 * 2 x N_b^2 x n_k c128 plus row buffers. KBE_ERR_OOM if it does not fit. */
kbe_status kbe_create(const kbe_config *cfg, void *stream, kbe_handle **out);
kbe_status kbe_destroy(kbe_handle *h);

/* h0_ab(k) = sum_r t_ab(R_r) exp(i k.R_r) (Sec. 2 band energies as hoppings).
 * R: host int [nhop][2] (R[r][1] ignored for dim 1); t: host c128
 * [nhop][nb][nb]. The resulting h0(k) must be Hermitian; not checked. */
kbe_status kbe_set_hamiltonian(kbe_handle *h, int nhop, const int *R, const double *t);

/* U(t_i) samples (len = nt_max + 1) or one constant (len = 1), the U(t) of
 * Eqs. 2 and 7; v: host double [nb][nb] pairing pattern v_ab, NULL keeps
 * the current one (default 1 - delta_ab, the paper's pair of bands). v must
 * be symmetric (the interaction U sum_ab v_ab n_a n_b of Eq. 2 is; an
 * asymmetric v would make the mean field non-Hermitian): KBE_ERR_ARG
 * otherwise. */
kbe_status kbe_set_interaction(kbe_handle *h, int len, const double *U, const double *v);

/* Peierls vector potential samples A_i = A(t_{i+1/2}), i < len (len >= 1), the
 * drive of step t_i -> t_{i+1}; dir: host double[dim] unit direction d.
 * A == NULL or len == 0 removes the drive. */
kbe_status kbe_set_drive(kbe_handle *h, int len, const double *A, const double *dir);

/* Dipole (length-gauge) drive of Eq. 4: during step t_i -> t_{i+1}, h(k) gains
 * E_i M, with E_i (host double, len samples) the step-averaged field and M
 * (host c128 [nb][nb], Hermitian, k-independent; the paper's two-band
 * d_k = 1 coupling is M = [[0,1],[1,0]]). A pulse I delta(t - t_p) is the
 * sample E_i = I / dt of the step that contains t_p. Steps beyond len use 0.
 * E == NULL or len == 0 removes the drive. Combines with the Peierls drive. */
kbe_status kbe_set_dipole(kbe_handle *h, int len, const double *E, const double *M);

/* t = 0: G^<(k;0,0) = i f(h0(k)), G^>(0,0) = G^<(0,0) - i, I = 0 (no initial
 * correlations). Clears a sticky error. Requires kbe_set_hamiltonian. */
kbe_status kbe_reset(kbe_handle *h);

/* Graph replay of kbe_step (enable != 0; off by default): the first
 * kbe_step(h, k) from a given row captures the kernels of those k steps into a
 * CUDA graph on the handle's stream, instantiates it and launches it; a later
 * call from the same row with the same k (e.g. after kbe_reset) launches the
 * instantiated graph, with no per-kernel launch cost. Results are identical to
 * the ordinary path. Any kbe_set_* call drops the cached graphs (captured
 * kernels carry the inputs by value). Needs a stream other than the legacy
 * default stream (otherwise steps run ungraphed); profiled steps run ungraphed. */
kbe_status kbe_set_graphs(kbe_handle *h, int enable);

/* Autotuner of the collision sweep's launch shape. The free parameter is the
 * split of the memory-time range over CTAs (how many CTAs share one output
 * column), expressed as the CTAs per SM the grid aims for. kbe_autotune times
 * candidate splits on this handle's buffers at one row per power-of-two bucket
 * of n (n + 1 in [2^b, 2^(b+1)), up to nt_max) and keeps the fastest per
 * (precision, quadrature, N_b, n_k, bucket) for the rest of the process; every
 * later sweep of that shape (any handle) uses it, untuned shapes keep the
 * default. For complex64 histories the candidates include the single-read
 * tile sweep (see kbe_set_sweep_choice). Only scratch buffers are written
 * (it may be called between steps);
 * cached graphs are dropped. targets (host int [KBE_AUTOTUNE_BUCKETS], may be
 * NULL) receives the choice per bucket (0: bucket above nt_max). Synchronises. */
#define KBE_AUTOTUNE_BUCKETS 17
kbe_status kbe_autotune(kbe_handle *h, int *targets);

/* TEST ONLY -- not for production use. Fault injection for testing the
 * failure path (no GPU fault, no hang):
 * KBE_INJECT_STAGED_COPY_LOSS makes the next collision sweep of this handle
 * (C64, staged form: N_b in {4, 8, 16}, n_k even) lose one CTA's first
 * copies. Its waits are bounded (one second of device time), so the kernel
 * marks a timeout and returns; the next synchronising call returns
 * KBE_ERR_TIMEOUT, which is sticky until kbe_reset. 0 clears. One-shot.
 * (If a timed-out kernel could not also drain its own copies in flight, the
 * handle is unusable: kbe_reset and kbe_checkpoint_load return KBE_ERR_STATE
 * and the handle must be destroyed and recreated.) */
#define KBE_INJECT_STAGED_COPY_LOSS 1
kbe_status kbe_debug_inject(kbe_handle *h, int fault);

/* Corrector passes run at each step 0..current (host int [n+1]; entry 0 is 0):
 * n_corr everywhere when corr_tol = 0. Synchronises. */
kbe_status kbe_corrector_iterations(kbe_handle *h, int *out);

/* Advance nsteps rows with P(EC)^n_corr E (Algorithm 1). Asynchronous on the
 * handle's stream. KBE_ERR_STATE past nt_max or before kbe_reset. */
kbe_status kbe_step(kbe_handle *h, int nsteps);

/* Wait for the handle's stream; returns the sticky device status. */
kbe_status kbe_synchronize(kbe_handle *h);

/* Index of the last completed row (-1 before kbe_reset). */
kbe_status kbe_current_step(const kbe_handle *h, int *n);

/* Equal-time observables at row `step` (0 <= step <= current): n_kb = Re rho_bb(k)
 * into host double [nk][nb] (may be NULL) and scalars[6] = {N, E_kin, E_HF,
 * E_corr, E_shift, E_tot} (may be NULL). Synchronises the stream. */
kbe_status kbe_observables(kbe_handle *h, int step, double *n_kb, double *scalars);

/* Observables of rows 0..current at once: n_kb host double [(n+1)][nk][nb]
 * and scalars host double [(n+1)][6] (either may be NULL). Synchronises. */
kbe_status kbe_observables_all(kbe_handle *h, double *n_kb, double *scalars);

/* Row i of G^x (which 0: lesser, 1: greater), blocks j = 0..i, into host c128
 * [(i+1)][nk][nb][nb]. Synchronises. */
kbe_status kbe_get_row(kbe_handle *h, int i, int which, double *out);

/* Device-pointer forms of kbe_observables_all and kbe_get_row, for callers
 * whose buffers live on the GPU (e.g. torch tensors): the same data and
 * layouts, written into caller-owned device memory of the current device.
 * The work is enqueued on the handle's stream and the call returns before it
 * completes (order later work after that stream or synchronise it). These
 * calls do not synchronise, so they do not read the sticky device status:
 * the next synchronising call (kbe_synchronize) reports it. */
kbe_status kbe_observables_all_dev(kbe_handle *h, double *n_kb_dev, double *scalars_dev);
kbe_status kbe_get_row_dev(kbe_handle *h, int i, int which, void *out_dev);

/* Collision-integral sweep timing (CUDA events around each sweep launch). */
kbe_status kbe_profile_enable(kbe_handle *h, int enable);
kbe_status kbe_profile_read(kbe_handle *h, kbe_profile_stats *out);

/* Checkpoint / resume. The state after row n is rows 0..n of the history,
 * the two FP64 working rows, the last collision row and the densities and
 * observables of rows 0..n; inputs (hoppings, interaction, drive) are not
 * part of it. kbe_checkpoint_bytes: size of the current state (0 before
 * kbe_reset). kbe_checkpoint_save copies it into caller-owned host memory of
 * that size (synchronises). kbe_checkpoint_load restores it into a handle
 * created with the same configuration (KBE_ERR_ARG otherwise); stepping then
 * continues from row n exactly as the saving handle would have, given the
 * same inputs. */
size_t kbe_checkpoint_bytes(const kbe_handle *h);
kbe_status kbe_checkpoint_save(kbe_handle *h, void *host, size_t bytes);
kbe_status kbe_checkpoint_load(kbe_handle *h, const void *host, size_t bytes);

/* Device bytes kbe_create would allocate for cfg (0 if cfg is invalid). */
size_t kbe_memory_bytes(const kbe_config *cfg);

/* ---------------------------------------------------------------------- */
/* reverse mode                                                             */
/* ---------------------------------------------------------------------- */

/* Gradient of a loss of the current row's occupations. The paper has no
 * counterpart: it only propagates (Algorithm 1). With N = the current step
 * and n_kb = Im G^<_bb(k; t_N, t_N) (the occupations kbe_observables
 * reports), given g = dL/dn_kb (host double [nk][nb]), returns
 *   dL_dA[i] = dL/dA_i for i < N (host double [nt_max]; entries >= N are 0),
 *              A_i being the Peierls sample the step to t_{i+1} used (the
 *              i-th kbe_set_drive sample, or its last one when fewer were
 *              given),
 *   dL_dU    = dL/dU: host double [1] for the constant U of
 *              kbe_set_interaction (len 1), or host double [nt_max + 1] with
 *              dL/dU(t_i) per sample when it was given U(t) samples (entries
 *              beyond t_N are 0),
 * the exact derivative of the computed trajectory (the discrete adjoint of
 * Algorithm 1 as this library evaluates it: the trapezoid collision sums, the
 * DFT form of Eq. 7, the series propagators, the mean field and the
 * predictor-corrector schedule). Steps are recomputed one at a time from the
 * stored history, so no per-step tape is kept; the history is left as it was
 * and stepping may continue afterwards.
 * Requires KBE_PREC_FP64, at least one step, and dt ||h(k)||_rowsum <= 1/4
 * at every step (the propagators' unscaled series); KBE_ERR_UNSUPPORTED
 * otherwise (the handle stays usable). The first call allocates
 * kbe_backward_memory_bytes(cfg) of device memory, kept until kbe_destroy
 * (KBE_ERR_OOM if it does not fit). Synchronises. */
kbe_status kbe_backward(kbe_handle *h, const double *dL_dn, double *dL_dA, double *dL_dU);
size_t kbe_backward_memory_bytes(const kbe_config *cfg);

/* ---------------------------------------------------------------------- */
/* batched systems (independent systems of uneven N_b, n_k, N_t)            */
/* ---------------------------------------------------------------------- */

typedef struct kbe_batch kbe_batch;

/* Create nsys independent systems. Each admitted system gets its own handle
 * on its own stream forked from `stream` (kernels of different systems run
 * concurrently). Systems are admitted in order while their memory
 * (kbe_memory_bytes) fits in budget_bytes (0: the device's free memory minus
 * 2 GiB); admitted (host int[nsys], may be NULL) receives 1 / 0 per system.
 * Systems that do not fit are not created: the caller may run them in a
 * later batch or with a smaller nt_max (each reported, never silent). */
kbe_status kbe_batch_create(int nsys, const kbe_config *cfgs, void *stream, size_t budget_bytes,
                            kbe_batch **out, int *admitted);
kbe_status kbe_batch_destroy(kbe_batch *b);
/* The handle of system i (NULL if i is out of range or was not admitted):
 * set its inputs and read its outputs with the handle API. */
kbe_handle *kbe_batch_system(kbe_batch *b, int i);
/* kbe_reset on every admitted system. */
kbe_status kbe_batch_reset(kbe_batch *b);
/* Advance every admitted system by nsteps rows (a system that reaches its
 * nt_max stops there), one time step of all systems at a time; work is
 * ordered after `stream`'s prior work and `stream` waits for all of it. */
kbe_status kbe_batch_step(kbe_batch *b, int nsteps);
/* Wait for all systems; the first failing system's status. */
kbe_status kbe_batch_synchronize(kbe_batch *b);
/* Graph mode for the batch. With a non-default stream, each kbe_batch_step(b, k)
 * runs the k steps of every admitted system as ONE captured graph launched on
 * that stream (each system's kernels on its own stream inside the graph):
 * captured on the first call with a given (rows, counts, ring order) shape,
 * replayed by later calls of the same shape, e.g. after kbe_batch_reset.
 * Changing a system's inputs (kbe_set_*, kbe_autotune) invalidates the
 * graph. On the default stream each system replays its own graph
 * (kbe_set_graphs). Results are bitwise those of the stream-ordered batch.
 * Synchronises the batch's stream. enable = 0 switches back. */
kbe_status kbe_batch_set_graphs(kbe_batch *b, int enable);
/* Persistent mode for the batch (FP64 histories only; KBE_ERR_UNSUPPORTED
 * otherwise, or while a system has profiling or an injected fault on). Each
 * kbe_batch_step runs the steps stage-major: every system advances on its own
 * stream up to its next collision sweep (Eq. 6, the memory integrals of the
 * predictor-corrector step of Sec. 3), then the sweeps of the systems of one
 * sweep class (N_b, quadrature, kernel form) run as ONE persistent launch per
 * lane (the systems of a class alternate between two lanes, each on its own
 * stream): the CTAs walk the concatenated block lists of the lane's systems,
 * each at its own autotuned l-split (kbe_autotune); then those systems
 * continue. A launch waits only for the systems of its own lane. With
 * graphs on (kbe_batch_set_graphs) and a non-default stream the call is one
 * captured graph as before. Results are bitwise those of the stream-ordered
 * batch. Synchronises the batch's stream; enable = 0 switches back. */
kbe_status kbe_batch_set_persistent(kbe_batch *b, int enable);
/* Persistent sweep launches that kbe_batch_step has enqueued in the eager
 * persistent mode (graph replays are not counted); -1 for a NULL batch. */
long kbe_batch_sweep_launches(const kbe_batch *b);

/* Diagnostics of the loaded library on the current device: binary_version
 * (may be NULL) receives the compute capability its kernels were compiled for
 * (cudaFuncGetAttributes; 103 for sm_103a), sm_count (may be NULL) the
 * device's streaming multiprocessors, against which grids are sized. */
kbe_status kbe_device_info(int *binary_version, int *sm_count);

/* Measured FMA throughput of the current device in GFLOP/s (2 flops per
 * FMA): FP64 (fp64_gflops) and FP32 (fp32_gflops), either may be NULL.
 * Grids of 4 and 8 CTAs per SM run 4, 8 or 16 independent FMA chains per
 * thread in two forms (accumulation with register operands; iteration),
 * timed with CUDA events on the default stream (best of three runs after a
 * warm-up each; the largest rate of the twelve configurations; takes a few
 * seconds and synchronises).
 * These are the denominators of the ALU-bound sweep forms' roofline
 * fractions: the FP64 form on the FP64 pipe, the double-float and complex64
 * forms on the FP32 pipe. Allocates and frees 8 bytes of device memory. */
kbe_status kbe_measure_fma_peaks(double *fp64_gflops, double *fp32_gflops);

/* Message of the last error of this handle; with NULL, of the last failed
 * create or handle-free operation (kbe_op_*) on the calling thread. */
const char *kbe_last_error(const kbe_handle *h);

/* ---------------------------------------------------------------------- */
/* stateless per-step operations on device buffers                          */
/*                                                                         */
/* Device layout: a "block" is one time pair (i, j) of both components,     */
/* c128 [2][nb][nb][nk] (component x = 0 lesser, 1 greater; k fastest). The */
/* history is the lower triangle, block (i, j), i >= j, at index             */
/* i(i+1)/2 + j. A "row" of m blocks is [m][2][nb][nb][nk]. Per-k matrices   */
/* are [nb][nb][nk]; per-k eigenvalues [nb][nk] doubles.                     */
/* ---------------------------------------------------------------------- */

typedef struct kbe_mesh {
  int nb;    /* bands (see kbe_config)           */
  int L[2];  /* mesh extents, L[1] = 1 for 1-D   */
} kbe_mesh;

/* The choice kbe_autotune stores, set by hand for one sweep shape (mesh m,
 * precision, quadrature) and row bucket (n + 1 in [2^bucket, 2^(bucket+1));
 * -1: every bucket), for every handle and stateless call of that shape:
 *   choice > 0 (<= 64): the per-column sweep, its l-split aiming at `choice`
 *                       CTAs per SM;
 *   choice < 0:         the single-read tile sweep (KBE_PREC_C64, N_b in
 *                       {2, 4, 8}, n_k even), TI = -choice rows per work
 *                       item (TI >= 32; an odd -choice means -choice - 1 rows
 *                       with one CTA per work unit instead of persistent CTAs
 *                       that claim units): each stored block is read from HBM
 *                       once and feeds both of its uses;
 *   choice = 0:         back to the built-in default (the tile sweep from
 *                       row 255 on where it applies).
 * The choice changes the summation order only. KBE_ERR_ARG if the choice does
 * not apply to the shape. kbe_autotune's targets use the same encoding. Not
 * thread safe against concurrent sweeps of the same shape. */
kbe_status kbe_set_sweep_choice(const kbe_mesh *m, int precision, int quadrature, int bucket, int choice);

/* (a1) Second-Born self-energy row, Eq. 7:
 *   Sigma^x(k; t_n, t_l), l = 0..n, from row n of G (blocks (n, l)),
 * computed as DFT_k -> real-space band products -> inverse DFT (exact
 * rewriting of the q, k' sums). v: host double [nb][nb] pairing pattern.
 * U(t_n) U(t_l) = Un * Ul_dev[l] (Ul_dev: device double [n+1]) or Un * Un if
 * Ul_dev is NULL. Grow_dev: row n, (n+1) blocks; Sigma_dev: (n+1) blocks.
 * work_dev: device scratch of kbe_op_sigma_row_workspace(m, n) bytes. */
size_t kbe_op_sigma_row_workspace(const kbe_mesh *m, int n);
kbe_status kbe_op_sigma_row(const kbe_mesh *m, const double *v, int n, double Un,
                            const double *Ul_dev, const void *Grow_dev, void *Sigma_dev,
                            void *work_dev, size_t work_bytes, void *stream);

/* Pack nblocks history blocks (device, FP64 [2][nb][nb][nk] = G^<, G^>;
 * block_elems = nb*nb*nk) into the history storage of a precision (device):
 * component 0 holds G^<, component 1 holds dG = G^< - G^> (formed in FP64),
 * as complex128 (FP64), float4 {re_hi, re_lo, im_hi, im_lo} with
 * hi = fl32(x), lo = fl32(x - hi) (DF64), or complex64 (C64). */
kbe_status kbe_op_pack(int precision, const void *src_dev, void *dst_dev, size_t nblocks,
                       size_t block_elems, void *stream);

/* kbe_op_pack for a history triangle of mesh m from row 0 (nblocks =
 * (n+1)(n+2)/2 for rows 0..n), in every precision including KBE_PREC_F16X2,
 * whose layout depends on N_b and n_k (kbe_op_pack refuses it with
 * KBE_ERR_UNSUPPORTED). dst_dev holds kbe_history_bytes(m, n, precision). */
kbe_status kbe_op_pack_mesh(const kbe_mesh *m, int precision, const void *src_dev, void *dst_dev,
                            size_t nblocks, void *stream);

/* Bytes of a history triangle with rows 0..n in a precision's storage:
 * (n+1)(n+2)/2 blocks of 2 nb^2 nk stored complex numbers (16 bytes each in
 * FP64 and DF64, 8 in C64); KBE_PREC_F16X2 (8 bytes per complex number) pads
 * every row to whole strips of 16 (N_b = 4) or 8 (N_b = 8) blocks. 0 if the
 * arguments are invalid. */
size_t kbe_history_bytes(const kbe_mesh *m, int n, int precision);

/* (a2) Collision-integral row, Eq. 6 in left form:
 *   I^x(n, j) = sum_{l=0}^{n} w^(n)_l [S^>(n,l) - S^<(n,l)] G^x(l, j)
 *             + sum_{l=0}^{j} w^(j)_l S^x(n,l) [G^<(l,j) - G^>(l,j)],
 * j = 0..n, with trapezoid weights w^(m)_l = dt (1 - [l=0]/2 - [l=m]/2)
 * (zero for m = 0) and G(l, j) = -G(j, l)^+ above the diagonal.
 * H_dev: history triangle with rows 0..n; Sigma_dev: n+1 blocks; I_dev:
 * n+1 blocks written (complex128). precision: KBE_PREC_*; H_dev holds the
 * triangle packed by kbe_op_pack in that precision's storage, Sigma_dev and
 * I_dev are complex128. work_dev: device scratch of
 * kbe_op_collision_row_workspace(m, n, precision) bytes (coefficient rows
 * and, when the l sum is split over CTAs, FP64 partial sums). */
size_t kbe_op_collision_row_workspace(const kbe_mesh *m, int n, int precision);
kbe_status kbe_op_collision_row(const kbe_mesh *m, int n, double dt, int precision,
                                const void *H_dev, const void *Sigma_dev, void *I_dev,
                                void *work_dev, size_t work_bytes, void *stream);

/* kbe_op_collision_row with the weights of `quadrature` (KBE_QUAD_*). */
kbe_status kbe_op_collision_row_quad(const kbe_mesh *m, int n, double dt, int precision, int quadrature,
                                     const void *H_dev, const void *Sigma_dev, void *I_dev,
                                     void *work_dev, size_t work_bytes, void *stream);

/* (a3) Step propagators of a Hermitian h(k) (device [nb][nb][nk] c128):
 * U = e^{-i dt h}, V = (U - 1) h^{-1} (= -i dt on the null space of h), each
 * device [nb][nb][nk] c128, by power series in dt / 2^s with doublings. */
kbe_status kbe_op_propagators(const kbe_mesh *m, double dt, const void *h_dev, void *U_dev,
                              void *V_dev, void *stream);

/* (a4) Row n from row n-1 (Algorithm 1, "solve Eq. 5"), given the step's
 * h, U = e^{-i dt h} and V = (U - 1) h^{-1} (per-k [nb][nb][nk] c128):
 *   G^x(n, j) = U G^x(n-1, j) + V Ibar^x(j),  j < n,
 *   Ibar = (1 - theta) I_{n-1}(j) + theta I_n(j),
 *   G^<(n, n) = U G^<(n-1, n-1) U^+ - i int_0^dt e^{-i h u} Sbar e^{i h u} du,
 *   Sbar = (1-theta)(I^<_{n-1}(n-1) + h.c.) + theta (I^<_n(n) + h.c.),
 *   G^>(n, n) = G^<(n, n) - i.
 * Gprev_dev: row n-1 (n blocks); Iprev_dev: n blocks; Icur_dev: n+1 blocks
 * (read only if theta != 0); out_dev: row n (n+1 blocks). n >= 1. U and V
 * must be h's propagators as kbe_op_propagators returns them: where dt ||h||
 * <= 1/4 (row-sum norm, the largest over the k-points the time diagonal
 * groups together) the diagonal takes U as given instead of forming it. */
kbe_status kbe_op_update_row(const kbe_mesh *m, int n, double dt, double theta, const void *h_dev,
                             const void *U_dev, const void *V_dev, const void *Gprev_dev,
                             const void *Iprev_dev, const void *Icur_dev, void *out_dev,
                             void *stream);

/* ---------------------------------------------------------------------- */
/* self-energy row without any allocation                                   */
/* ---------------------------------------------------------------------- */

/* Size of the device array that kbe_op_sigma_row_noalloc uses as scratch. */
#define KBE_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* Same operation, arguments, layouts and result as kbe_op_sigma_row, minus
 * the workspace arguments; the paper has no counterpart (it is a service for
 * callers that cannot allocate device memory: hosts whose device memory is
 * all owned by their own allocator, loops where cudaMalloc/cudaFree would
 * synchronise the device, plug-ins with a fixed memory budget).
 * Scratch: one file-scope device array of KBE_NOALLOC_SCRATCH_BYTES inside
 * libkbe, resident on every GPU that loads the library until the process
 * exits. The call allocates and frees nothing.
 * Limit: the row must need at most KBE_NOALLOC_SCRATCH_BYTES of scratch
 * (kbe_op_sigma_row_workspace(m, n) bytes); larger rows are rejected with
 * KBE_ERR_ARG and a message in kbe_last_error(NULL), before any GPU work.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins. The address is then kept for the life of
 * the process: after cudaDeviceReset (or anything else that destroys the
 * device's primary context) it is stale, so do not call this entry point
 * again in that process.
 * Sharing: all calls use the same array and it keeps the last call's
 * contents (no call depends on them); calls whose GPU work overlaps, e.g. on
 * two streams or from two host threads, race on it and must be serialised by
 * the caller. */
kbe_status kbe_op_sigma_row_noalloc(const kbe_mesh *m, const double *v, int n, double Un,
                                    const double *Ul_dev, const void *Grow_dev, void *Sigma_dev,
                                    void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KBE_H */
