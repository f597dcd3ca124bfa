/*
 * ystat -- power-spectrum multipoles P_0, P_2, P_4 of a galaxy survey with a varying
 * line of sight, by the FFT-based Yamamoto estimator of Bianchi, Gil-Marin, Ruggeri &
 * Percival (2015), on one NVIDIA GB300 (sm_103a).
 *
 * The calls follow the paper's statement of the problem:
 *   Eq. (1)       F(r) = w(r) [n(r) - alpha n_s(r)] / I^(1/2)     -> ys_assign
 *   Eqs. (4)-(13) P_l(k) from A_0, B_ij, C_ijl via FFTs             -> ys_measure_multipoles
 * All arithmetic runs in the CUDA kernels of this library; there is no CPU fallback.
 * A call that needs the GPU fails with YS_ERR_CUDA when no usable device is present.
 *
 * Conventions shared by every call
 *  - Positions are comoving Cartesian coordinates (Mpc/h), float32, structure of
 *    arrays.  The analysis box is the cube [box_min, box_min + box_len)^3, divided into
 *    n_mesh^3 cells of side H = box_len / n_mesh; mesh node i sits at box_min + i H
 *    (the interlaced mesh at box_min + (i + 1/2) H).  The box is periodic.
 *  - Pointers named d_* are device pointers, h_* host pointers.  The caller owns every
 *    buffer it passes; no call keeps a caller pointer after it returns.
 *  - Work is queued on the plan's CUDA stream and is asynchronous unless a call says
 *    otherwise.  Calls on one plan must not overlap.
 *  - Every call returns a ys_status and never aborts the process.
 */
#ifndef YSTAT_H
#define YSTAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  YS_OK = 0,
  YS_ERR_ARG = 1,          /* invalid argument, or particles outside the box   */
  YS_ERR_OOM = 2,          /* device allocation failed                          */
  YS_ERR_CUDA = 3,         /* CUDA runtime error (see ys_last_cuda_error)       */
  YS_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out                */
  YS_ERR_UNSUPPORTED = 5,  /* mesh size or option this build does not handle   */
  YS_ERR_STATE = 6         /* call out of order (e.g. measure before assign)    */
} ys_status;

typedef enum { YS_NGP = 1, YS_CIC = 2, YS_TSC = 3 } ys_assign_kind;

/* Estimator configuration.
 *  n_mesh     N: 16 <= N <= 1024, N = 2^a or 3 * 2^a (a >= 4 for the latter).
 *  box_min, box_len, observer   geometry; r = node - observer is the line of sight
 *             used for the LOS weights of Eqs. (11) and (13) (weight 0 at r = 0).
 *  assign     NGP / CIC / TSC particle-to-mesh kernel (Sec. 4 uses CIC).
 *  interlace  1: a second mesh shifted by H/2 on every axis; the two transforms are
 *             averaged with the phase e^{-i k.(H/2)(1,1,1)}.
 *  compensate 1: divide every A_n(k) by prod_i sinc(k_i H / 2)^p, p = 1, 2, 3.
 *  ell_max    0, 2, 4 or 6: highest multipole; 1, 7 or 22 fields of Sec. 3 for l <= 4.
 *             6 is the same decomposition one order up (the paper notes after Eq. 13
 *             that higher orders follow alike): 28 more fields F r_i..r_n / r^6, and
 *             P_6 = 13/I <Re A_0 A_6^*> - the l = 6 term of Eq. (4).  l_max = 6 is
 *             supported for N <= 512 (YS_ERR_UNSUPPORTED above).
 *  k_min, dk, n_bins   shells [k_min + b dk, k_min + (b+1) dk), b < n_bins <= 4096; only
 *             modes with 0 < |k| < k_Nyquist = pi N / box_len enter.  The x stage holds
 *             every shell's sums in shared memory (24 bytes per shell at the least);
 *             every supported mesh fits 4096 shells, and ys_plan_create returns
 *             YS_ERR_UNSUPPORTED (ys_last_cuda_error() says why) for a device whose
 *             shared memory per block is too small.
 *  alpha      < 0: alpha = sum_gal w / sum_ran w (Eq. 1); else this value.
 *  max_particles   capacity (galaxies + randoms) of the plan's particle buffers.
 *  stream     cudaStream_t to queue work on (NULL = legacy default stream). */
typedef struct {
  int32_t n_mesh;
  double box_min[3];
  double box_len;
  double observer[3];
  int32_t assign;
  int32_t interlace;
  int32_t compensate;
  int32_t ell_max;
  double k_min;
  double dk;
  int32_t n_bins;
  double alpha;
  int64_t max_particles;
  void* stream;
} ys_config;

/* A catalogue: n particles, float32 arrays of length n.
 * w    NULL = unit weights.  nbar: expected galaxy density at each position (Eq. 1),
 * used for the normalisation I (randoms only); NULL = not given (I is then 0 and
 * P_l are NaN).  Device pointers for ys_assign, host pointers for ys_estimate_host. */
typedef struct {
  const float* x;
  const float* y;
  const float* z;
  const float* w;
  const float* nbar;
  int64_t n;
} ys_catalog;

/* Host-side result of one measurement (arrays of length n_bins, caller-owned).
 * k_mean  mean |k| of the modes in the shell (h/Mpc); n_modes  number of modes (full
 * k-space count); p0, p2, p4  the multipoles of Eqs. (6)-(8) in (Mpc/h)^3 with the
 * shot noise S/I subtracted from p0 only (Eq. 3).  Empty shells give NaN and
 * n_modes = 0.  Any array pointer may be NULL.  alpha, norm_I = alpha sum_ran w^2 nbar,
 * shot_noise = S / I with S = sum_gal w^2 + alpha^2 sum_ran w^2 are filled in.
 * p6 receives P_6 for l_max = 6 plans (NaN otherwise). */
typedef struct {
  double* k_mean;
  double* n_modes;
  double* p0;
  double* p2;
  double* p4;
  double alpha;
  double norm_I;
  double shot_noise;
  double* p6;
} ys_result;

typedef struct ys_plan_s ys_plan;

/* Validate cfg and create a plan: allocates the meshes, the transformed fields,
 * the shell tables and the particle buffers on the current device (cudaMalloc);
 * the plan owns and frees them.  Host-side; may synchronise the device. */
ys_status ys_plan_create(const ys_config* cfg, ys_plan** out);

/* Device bytes the plan holds (0 if plan is NULL). */
size_t ys_plan_device_bytes(const ys_plan* plan);

/* Eq. (1): deposit galaxies (+w) and randoms (-alpha w) onto the mesh(es), and
 * accumulate the FP64 catalogue sums behind alpha, I and S.  gal/ran hold DEVICE
 * pointers.  Asynchronous.  Particles outside the box are wrapped periodically and
 * reported by the next ys_measure_multipoles as YS_ERR_ARG. */
ys_status ys_assign(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran);

/* Shared randoms.  Sec. 4 notes that catalogues which share one random catalogue
 * (mocks measured against the same randoms) need it processed only once.
 * ys_randoms_cache deposits ran (DEVICE pointers) once, with weight +w, into a
 * plan-owned copy of the mesh(es) -- an extra m n_mesh^3 floats, allocated on the
 * first call -- and keeps the FP64 sums sum w, sum w^2, sum w^2 nbar.  It overwrites
 * the plan's current assignment (call ys_assign or ys_assign_cached again before
 * measuring).  Asynchronous. */
ys_status ys_randoms_cache(ys_plan* plan, const ys_catalog* ran);

/* Eq. (1) against the kept randoms: deposits gal (DEVICE pointers) only and writes
 * F = (galaxy deposit) - alpha (kept random deposit), alpha = sum_gal w / sum_ran w
 * (or cfg.alpha) formed on the device, with the catalogue sums of I and S completed
 * from the kept ones.  The result equals ys_assign with the same randoms up to float
 * rounding.  YS_ERR_STATE without a ys_randoms_cache.  Asynchronous. */
ys_status ys_assign_cached(ys_plan* plan, const ys_catalog* gal);

/* The assigned mesh F of Eq. (1), as the transforms read it: m meshes of n_mesh^3
 * floats (m = 2 when interlaced; the second has its nodes at +H/2 on every axis),
 * each x-major with z fastest.  Copies the m n_mesh^3 floats to dst, a DEVICE or HOST
 * pointer owned by the caller, on the plan's stream and waits for the copy.  With
 * the sorted assignment each node is summed exactly in fixed point (every stencil
 * weight rounded to 2^-s, s set per tile from its largest |w| and its record count,
 * far below float resolution), so the mesh does not depend on the order of the
 * particles; tiles with a non-finite weight, tile shapes that do not fit twice in
 * shared memory, and the direct assignment sum in float.
 * YS_ERR_ARG for a null pointer or count < m n_mesh^3, YS_ERR_STATE before an
 * assignment. */
ys_status ys_plan_copy_mesh(ys_plan* plan, float* dst, int64_t count);

/* Eqs. (4)-(13): the LOS-weighted fields, their FFTs, the k-space combination,
 * the shell sums and Eqs. (6)-(8).  Writes the device result row
 *   d_out[0 .. 5 n_bins + 5) = [k_mean | n_modes | p0 | p2 | p4 |
 *                              alpha, I, S/I, particles outside the box, timeout flag]
 * (doubles), followed for l_max = 6 by p6 in d_out[5 n_bins + 5 .. 6 n_bins + 5),
 * asynchronously.  d_out may be NULL (the plan keeps its own copy). */
ys_status ys_measure_multipoles_async(ys_plan* plan, double* d_out);

/* As ys_measure_multipoles_async, then waits for the stream and copies the result
 * into the caller's host arrays.  Returns YS_ERR_TIMEOUT if a bounded device-side
 * wait ran out (results invalid), else YS_ERR_ARG if ys_assign saw particles
 * outside the box (results are still written). */
ys_status ys_measure_multipoles(ys_plan* plan, ys_result* out);

/* End-to-end convenience: gal/ran hold HOST pointers (pinned or pageable); copies them
 * to plan-owned device buffers, runs ys_assign and ys_measure_multipoles, and fills
 * the host result.  The copies run on the plan's stream and on three internal copy
 * streams at once (joined with events before the assignment); the galaxies' nbar is
 * not copied (only the randoms' enters I).  Synchronous. */
ys_status ys_estimate_host(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran,
                           ys_result* out);

/* Wedges P_perp (0 <= mu <= 1/2) and P_para (1/2 < mu <= 1) from the multipoles,
 * Sec. 5, Eqs. 16-17: P_perp = P_0 - 3/8 P_2 + 15/128 P_4 and
 * P_para = P_0 + 3/8 P_2 - 15/128 P_4, shell by shell (NaN where the shell has no
 * modes, and meaningful for l_max = 4 plans).
 * d_rows: n_cat result rows (DEVICE, layout of ys_measure_multipoles_async) spaced
 * `stride` doubles apart (>= 5 n_bins + 5).  d_out (DEVICE, caller-owned): n_cat x
 * [P_perp(n_bins) | P_para(n_bins)] doubles.  Asynchronous on stream (cudaStream_t,
 * NULL = legacy stream). */
ys_status ys_wedges(const double* d_rows, int32_t n_cat, int64_t stride, int32_t n_bins, double* d_out,
                    void* stream);


/* Sec. 4's "sum-gal": the estimator as a direct sum over galaxies and randoms,
 *   A_n(k) = sum_p s_p w_p (k_hat . r_hat_p)^n e^{-i k.x_p},  s = +1 (galaxies), -alpha (randoms),
 * r_p = x_p - observer the particle's own line of sight, at every half-grid mode
 * k = k_F m (k_F = 2 pi / box_len; m_x, m_y in [-n_mesh/2, n_mesh/2), m_z in
 * [0, n_mesh/2], weight 2 for 0 < m_z < n_mesh/2) with 0 < |k| < k_F n_mesh / 2 that
 * falls in a shell, then Eqs. (6)-(8) (and P_6 for l_max = 6).  No mesh, window or
 * aliasing: n_mesh only sets the k lattice (any even value 4..16384, not only FFT
 * sizes), so the sum reaches beyond any mesh's Nyquist frequency.  Its cost is
 * (galaxies + randoms) x modes, for small cases and as the reference the paper
 * compares the FFT method with.
 * cfg: n_mesh, box_min, box_len, observer, ell_max, k_min, dk, n_bins, alpha, stream are
 * used (assign, interlace, compensate, max_particles are ignored).  gal, ran: DEVICE
 * pointers, as for ys_assign.  d_out (DEVICE): one result row in the layout of
 * ys_measure_multipoles_async (its last two scalars are 0).  d_wedges (DEVICE, may be
 * NULL): [P_perp(n_bins) | P_para(n_bins)] by the wedges' definition, Sec. 5
 * Eqs. 14-15 in the Yamamoto form: the top hat Theta(|k_hat . r_hat_p| <= 1/2) on
 * one particle of each pair in place of L_l, normalised by 1 / (1/2), minus S/I.
 * Allocates scratch (cudaMalloc) and waits for the stream: synchronous. */
ys_status ys_sum_gal(const ys_config* cfg, const ys_catalog* gal, const ys_catalog* ran, double* d_out,
                     double* d_wedges);

/* Sec. 4's "sum-grid": the same direct sum over the nodes of the plan's assigned
 * mesh(es) (after ys_assign), each node carrying F with r = node - observer as in the
 * FFT path; an interlaced pair is averaged (nodes at +H/2 on the second mesh) and,
 * if the plan compensates, the window is divided out.  It is the exact DFT of what
 * the FFT path transforms, at the plan's modes and shells: the two agree shell by
 * shell to float rounding.  Cost: filled nodes x modes (any mesh, for a few thousand
 * modes; the nodes go through in chunks of 2^26, with 2 GB of scratch).
 * d_out, d_wedges as for ys_sum_gal.  YS_ERR_STATE before ys_assign.  Synchronous. */
ys_status ys_sum_grid(ys_plan* plan, double* d_out, double* d_wedges);

/* Per-kernel statistics (measurement support; no counterpart in the paper).
 * With profiling on, every kernel launch of the plan is bracketed by CUDA events on
 * the plan's stream and ys_measure_multipoles* launches directly instead of
 * replaying its captured CUDA graph.  Kernel classes, in order:
 *   0 particle count + catalogue sums, 1 tile scan, 2 particle binning,
 *   3 tile deposit, 4 y,z stage (LOS fields, FFTs along z and y, k_x-power grouping;
 *   one persistent launch), 5 (unused), 6 x-stage (FFT along x + combine + shells),
 *   7 finalize.
 * launches[c] counts kernel launches of class c, ms[c] their summed device time
 * (valid only for launches made while profiling was on). */
#define YS_NUM_KERNEL_CLASSES 8
typedef struct {
  int64_t launches[YS_NUM_KERNEL_CLASSES];
  double ms[YS_NUM_KERNEL_CLASSES];
} ys_stats;

/* enable != 0 turns event profiling on.  Host-side. */
ys_status ys_plan_set_profiling(ys_plan* plan, int enable);

/* Waits for the plan's stream, then fills *out with the counts and times since the
 * last reset; reset != 0 clears them afterwards. */
ys_status ys_plan_get_stats(ys_plan* plan, ys_stats* out, int reset);

/* Failure-path test hook (no counterpart in the paper).  Every wait of the y,z stage
 * (the persistent kernel of ys_measure_multipoles*) is bounded; when one runs out the
 * kernel stops, the call reports YS_ERR_TIMEOUT and the next measurement on the plan
 * starts clean.  This call shortens that bound and can make one wait run out on
 * purpose, so that the path can be exercised without any fault:
 *  wait_limit_ns  bound of each wait in ns (<= 0: the default, 1 s; at most 10 s).
 *  skip_plane     -1: normal operation.  0 <= skip_plane < m N (m = 2 when interlaced):
 *                 the row items of that x-plane finish their work but withhold their
 *                 completion signal, so the column items waiting for it time out.
 * Waits for the plan's stream, and drops the plan's captured measurement graph (the
 * next measurement captures it again with these settings).  YS_ERR_ARG for values
 * out of range. */
ys_status ys_plan_set_fault_injection(ys_plan* plan, int64_t wait_limit_ns, int32_t skip_plane);

/* ys_assign without any device allocation.  (The paper has no counterpart; this is
 * a deployment variant of the assignment step.)
 *
 * ys_assign keeps its sorting scratch -- per-tile counters and one record per
 * (particle, mesh tile it touches) -- in plan-owned buffers sized to the largest
 * catalogue seen, and grows them with cudaMalloc when a larger one arrives.  Callers
 * that must not allocate device memory after set-up (a fixed memory pool, an
 * embedding framework that owns every allocation, code that must not synchronise
 * the device the way cudaMalloc/cudaFree can) use this entry point instead: it takes
 * that scratch from one static device array of YS_NOALLOC_SCRATCH_BYTES (64 MiB) that
 * every GPU loading the library holds until the process exits, and calls no
 * cudaMalloc, cudaFree or other allocating routine.  The plan must already exist
 * (ys_plan_create allocates the mesh it writes; max_particles may be 0).
 *
 * Inputs: gal, ran with DEVICE pointers, as for ys_assign.  Output: the plan's mesh(es)
 * and catalogue sums, consumed by the next ys_measure_multipoles*.  Asynchronous on
 * the plan's stream.
 * Limits: the records need (gal->n + ran->n) * T * 16 bytes, T = 2^(axes with more
 * than one tile in the plan's current scatter-tile shape) <= 8 -- 16 x 16 x 16 nodes
 * unless ys_plan_autotune picked another shape -- plus 12 bytes per tile; a catalogue
 * that does not fit returns YS_ERR_UNSUPPORTED before any work is queued
 * (ys_last_cuda_error() then gives the sizes).  For a 256^3 mesh (T = 8) this is
 * about 520 000 particles.
 * Set-up: the first call on each device (and the first after that device's context
 * changed, e.g. after cudaDeviceReset) looks up the array's device address with
 * cudaGetSymbolAddress while that device is current; make that first call before
 * any stream capture.
 * Sharing: every call, on every plan, uses the same array and leaves its contents
 * behind; each call zeroes the counters it needs itself.  Calls whose work overlaps
 * on the GPU (different streams, different host threads) race on the array and must
 * be serialised by the caller. */
#define YS_NOALLOC_SCRATCH_BYTES (64u << 20)
ys_status ys_assign_noalloc(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran);

/* Free everything the plan owns.  NULL is accepted. */
ys_status ys_plan_destroy(ys_plan* plan);

/* ---- Autotuning and batched runs (throughput arrangements; no counterpart in the
 * paper's equations, which these calls evaluate unchanged) ---- */

/* Launch shapes the autotuner chose: scatter tile (nodes per axis; 0 0 0 = the direct
 * assignment, see ys_plan_set_direct_assign), CTAs of the persistent y,z kernel, the
 * lead (in x-planes) of its column items over its row items, and the x stage's FFT
 * tile (pencils transformed together by one CTA), with the best measured times. */
typedef struct {
  int32_t tile[3];
  int32_t yz_grid;
  int32_t ring_lead;
  double assign_ms;
  double measure_ms;
  int32_t x_pencils;
} ys_tuning;

/* Time the candidate scatter tiles (16x16x32, 8x16x32, 16x16x16, 32x16x32, 8x8x32)
 * and, for small meshes, the direct assignment; then the y,z grids (resident, 3/4,
 * 1/2), ring leads (0.7x, 1x, 1.4x, 2x a work-balanced estimate) and x-stage tiles
 * (the mesh's default pencils per CTA and half or twice that) on this catalogue
 * (DEVICE pointers), reps timed calls each, and keep the fastest in the plan.  Leaves
 * the catalogue assigned.  Synchronous.  out may be NULL. */
ys_status ys_plan_autotune(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran, int32_t reps,
                           ys_tuning* out);

/* Choose the assignment's arrangement (Eq. 1 either way): enable != 0 selects the
 * direct assignment, which reads each catalogue twice (its weights for alpha, I and
 * S, then its particles) and adds every stencil weight into the zeroed mesh with
 * global float reductions that stay in L2 -- offered when the plan's meshes hold at
 * most 64 MB (YS_ERR_UNSUPPORTED above); 0 selects the tile-sorted assignment (the
 * default).  ys_plan_autotune sets it by timing both.  Host-side. */
ys_status ys_plan_set_direct_assign(ys_plan* plan, int enable);

typedef struct ys_batch_s ys_batch;

/* Many catalogues -- the Sec. 1 use case of hundreds of mocks -- in one graph launch.
 * cfgs[i] configures catalogue i (its max_particles must bound gal_i.n + ran_i.n; its
 * stream is ignored).  Catalogues with the same configuration form a class, measured
 * in waves of up to `lanes` catalogues (1..32, at most 8 are used): each catalogue of
 * a wave is assigned on its own plan (lane), then one persistent y,z launch serves
 * every item of the whole wave through one work queue, one x-stage launch covers all
 * their pencil blocks and one launch finalizes their rows.  A class with more than
 * one wave holds up to four sets of min(lanes, its catalogues) plans on their own
 * streams and sends its waves round them (one wave assigns while another
 * transforms); the 8 streams are shared out among the classes.  Plans are sized for the class's largest
 * catalogue.  Host-side. */
ys_status ys_batch_create(const ys_config* cfgs, int32_t n, int32_t lanes, ys_batch** out);

/* Doubles between consecutive result rows of ys_batch_run: the longest row of the
 * batch (5 n_bins + 5, plus n_bins for l_max = 6 plans). */
int64_t ys_batch_result_stride(const ys_batch* batch);

/* Autotune each class on its largest catalogue (DEVICE pointers, arrays of n): the
 * launch shapes are chosen on one lane and given to the class's other lanes.
 * Synchronous. */
ys_status ys_batch_autotune(ys_batch* batch, const ys_catalog* gal, const ys_catalog* ran, int32_t reps);

/* Run the whole batch.  gal, ran: host arrays of n catalogues holding DEVICE pointers.
 * Row i of d_results (DEVICE, n x stride doubles) receives catalogue i's result row in
 * the layout of ys_measure_multipoles_async.  The first call, and any call whose
 * catalogue pointers, sizes or d_results differ from the last capture, captures the
 * batch into a CUDA graph (host-side work); later calls only launch it on `stream`
 * (cudaStream_t, NULL = legacy stream).  Asynchronous otherwise. */
ys_status ys_batch_run(ys_batch* batch, const ys_catalog* gal, const ys_catalog* ran, double* d_results,
                       void* stream);

/* Free the batch and its plans.  NULL is accepted. */
ys_status ys_batch_destroy(ys_batch* batch);

/* ---- Learned aliasing/window correction (no counterpart in the paper: the paper
 * notes that mesh aliasing is what separates its FFT estimate from the galaxy sum at
 * high k, and this network estimates that residual from a coarse measurement) ----
 *
 * Network: x (5) -> 64 -> 64 -> 64 -> 3, GELU (erf form) after each hidden layer,
 * linear output.  Parameters are a flat float vector of YS_MLP_PARAMS values,
 * row-major weights W[out][in] then bias for each layer in order:
 *   W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[3][64] b4[3].
 * The kernels use a bfloat16 copy of the weights (round to nearest even) and FP32
 * activations and accumulation; Adam updates an FP32 master copy.
 *
 * Per-shell features of a result row (layout of ys_measure_multipoles_async), with
 * D = P_0 + S/I the coarse monopole before shot-noise subtraction:
 *   x = [ k_mean / k_nyq, ln(D / (S/I)), P_2 / D, P_4 / D, (S/I) / D ]
 * Targets, given a fine-mesh row of the same catalogue and binning:
 *   t_l = (P_l^fine - P_l^coarse) / D,  l = 0, 2, 4.
 * Correction: P_l <- P_l + D y_l for every shell with modes.
 * Row layout of X: rows x 5 floats; of Y and T: rows x 3 floats (DEVICE). */
#define YS_MLP_PARAMS 8899
typedef struct ys_mlp_s ys_mlp;

/* Create a network on the current device from h_params (HOST, YS_MLP_PARAMS floats);
 * Adam moments start at zero.  Synchronous. */
ys_status ys_mlp_create(const float* h_params, ys_mlp** out);

/* Copy the FP32 master parameters, and optionally the Adam moments m, v (HOST,
 * YS_MLP_PARAMS floats each, may be NULL) and the step count, to the host.
 * Synchronous. */
ys_status ys_mlp_get_state(ys_mlp* mlp, float* h_params, float* h_m, float* h_v, int64_t* h_step);

/* Restore a state saved by ys_mlp_get_state (h_m, h_v NULL: zero moments). */
ys_status ys_mlp_set_state(ys_mlp* mlp, const float* h_params, const float* h_m, const float* h_v, int64_t step);

/* Y = net(X) for `rows` rows (DEVICE pointers).  Asynchronous on stream. */
ys_status ys_mlp_forward(ys_mlp* mlp, const float* d_x, int64_t rows, float* d_y, void* stream);

/* Gradient of loss = sum over rows and outputs of (y - t)^2 / (3 rows) with respect
 * to the parameters, at the bfloat16 weights, into d_grad (DEVICE, YS_MLP_PARAMS
 * floats, may be NULL) and the summed squared error into d_sse (DEVICE, one double,
 * may be NULL).  rows >= 1.  Asynchronous. */
ys_status ys_mlp_gradient(ys_mlp* mlp, const float* d_x, const float* d_t, int64_t rows, float* d_grad,
                          double* d_sse, void* stream);

/* One full-batch Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * the gradient above; refreshes the bfloat16 copy.  d_sse as above.  Asynchronous. */
ys_status ys_mlp_train_step(ys_mlp* mlp, const float* d_x, const float* d_t, int64_t rows, float lr,
                            double* d_sse, void* stream);

/* Features (and, if d_fine_rows != NULL, targets) of n_cat result rows spaced
 * `stride` doubles apart (DEVICE).  A shell enters when it has modes and finite
 * multipoles; d_src[j] = catalogue * n_bins + shell of feature row j and *d_count =
 * number of rows written (DEVICE int32; the order of rows is not fixed).  d_x needs
 * n_cat n_bins x 5 floats, d_t n_cat n_bins x 3, d_src n_cat n_bins.  Asynchronous. */
ys_status ys_mlp_features(const double* d_rows, const double* d_fine_rows, int32_t n_cat, int64_t stride,
                          int32_t n_bins, double k_nyq, float* d_x, float* d_t, int32_t* d_src, int32_t* d_count,
                          void* stream);

/* Corrected result rows: d_out (DEVICE, same layout; may equal d_rows) receives
 * d_rows with P_l + D y_l in every shell with modes.  Asynchronous; the first call
 * for a larger n_cat * n_bins allocates feature scratch. */
ys_status ys_mlp_correct(ys_mlp* mlp, const double* d_rows, int32_t n_cat, int64_t stride, int32_t n_bins,
                         double k_nyq, double* d_out, void* stream);

/* Free the network.  NULL is accepted. */
ys_status ys_mlp_destroy(ys_mlp* mlp);

/* Static description of a status code. */
const char* ys_status_string(ys_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* ys_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* YSTAT_H */
