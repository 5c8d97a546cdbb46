/*
 * dm.h -- C ABI of the GB300 multi-mode difference-map (DM) ptychography
 * library.
 *
 * One DM iteration (arXiv 1808.10375, Sec. II) over all views j and probe
 * modes k, with one object mode:
 *   Eq. 3   psi_j^k <- psi_j^k + beta ( F^-1 F_c[2 P_k O - psi_j^k] - P_k O )
 *           where F_c rescales every mode of its argument's transform by
 *           sqrt(I_j(q) / sum_k |F[.]_k(q)|^2), keeping the phase;
 *   Eq. 5   O(r)   <- sum_jk conj(P_k(r-r_j)) psi_j^k(r-r_j) / sum_jk |P_k(r-r_j)|^2
 *   Eq. 4   P_k(u) <- sum_j conj(O(r_j+u)) psi_j^k(u) / sum_j |O(r_j+u)|^2
 *   Eq. 6   relative change of O and of each P_k between iterations.
 *
 * Conventions fixed by this library (the paper leaves them open):
 *  - F is the orthonormal 2-D DFT with the zero frequency at [0][0]; where
 *    sum_k |F[.]_k(q)|^2 is zero the projected field is zero; negative
 *    intensities are rejected at dm_init.
 *  - Eq. 5 is applied first (with the probe the Fourier step used), then
 *    Eq. 4 with the new object (Gauss-Seidel), n_inner times per iteration.
 *  - Each overlap denominator gets delta = denom_floor_rel * max(denominator);
 *    object pixels that no view covers keep their value.
 *  - The Fourier error is E_F = sqrt(sum_jq (sqrt(S_j(q)) - sqrt(I_j(q)))^2 /
 *    sum_jq I_j(q)), S_j the mode sum of the Fourier step.
 *
 * Layouts (all row-major, complex = interleaved float pairs (re, im)):
 *   positions    int32  [J][2]        top-left (row, col) of each N x N footprint,
 *                                     0 <= row <= obj_h - N, 0 <= col <= obj_w - N
 *   intensities  float  [J][N][N]     recorded I_j(q), q = (qy, qx), DC at [0][0]
 *   probe        float  [M][N][N][2]  probe modes P_k(u)
 *   object       float  [H][W][2]     object O(r)
 *   exit waves   float  [J][M][N][N][2]
 *
 * Memory: every pointer argument is a host pointer when its mem_kind is
 * DM_HOST and a device pointer (on the context's device) when DM_DEVICE.
 * Inputs are copied at the call; the caller keeps ownership of every buffer
 * it passes.  All device memory the context needs is obtained once in
 * dm_init, through params->alloc (if non-NULL) or cudaMallocAsync on the
 * context's stream, and released by dm_free.
 *
 * Streams and synchronisation: all work is enqueued on params->stream (or a
 * stream the library creates when it is NULL).  dm_iterate only enqueues;
 * errors raised on the device (non-finite metrics, expired bounded waits)
 * are reported by the next call that synchronises: dm_sync, dm_get_*.
 *
 * Errors: every int-returning call returns DM_OK (0) or a negative DM_E*
 * code and never aborts; dm_last_error gives the message.  A context is not
 * thread-safe; distinct contexts are independent.
 */
#ifndef PTYCHO_DM_H
#define PTYCHO_DM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DM_OK 0
#define DM_EINVAL (-1)      /* bad shape, size, position, pointer or input value */
#define DM_ENOMEM (-2)      /* an allocation failed */
#define DM_ECUDA (-3)       /* a CUDA runtime error (text in dm_last_error) */
#define DM_ENONFINITE (-4)  /* a metric of some iteration was NaN or Inf */
#define DM_ETIMEOUT (-5)    /* a bounded device-side wait expired */

#define DM_HOST 0
#define DM_DEVICE 1

/* Steps for dm_run_step (one piece of an iteration, for per-step checks). */
#define DM_STEP_FOURIER 0   /* Eq. 3 over all views                          */
#define DM_STEP_OBJECT 1    /* Eq. 5 from the current exit waves and probe   */
#define DM_STEP_PROBE 2     /* Eq. 4 from the current exit waves and object  */

/* Kernel classes reported by dm_get_timing. */
#define DM_KERNEL_FOURIER 0       /* persistent Fourier-step kernel (Eq. 3)       */
#define DM_KERNEL_OBJECT_GATHER 1 /* object numerator/denominator gather (Eq. 5) */
#define DM_KERNEL_OBJECT_FINAL 2  /* object division and Eq. 6 partials          */
#define DM_KERNEL_PROBE_PARTIAL 3 /* per-view-group probe sums (Eq. 4)           */
#define DM_KERNEL_PROBE_FINAL 4   /* probe reduction, division, Eq. 6 partials   */
#define DM_KERNEL_METRICS 5       /* Eq. 6 / Fourier-error reductions            */
#define DM_KERNEL_OTHER 6         /* object-source refresh for n_inner > 1, etc. */
#define DM_KERNEL_COUNT 7

typedef struct dm_ctx dm_ctx;

/* Device allocator hook: return `bytes` of device memory on the context's
 * device (NULL on failure); free it again.  `user` is alloc_user. */
typedef void* (*dm_alloc_fn)(size_t bytes, void* user);
typedef void (*dm_free_fn)(void* ptr, void* user);

typedef struct dm_params {
  int32_t n;                  /* frame side N: 16, 32, 64, 128 or 256            */
  int32_t modes;              /* probe modes M, 1..16                            */
  int32_t views;              /* scan points J >= 1                              */
  int32_t obj_h, obj_w;       /* object array H x W, each >= N                   */
  float beta;                 /* Eq. 3 relaxation, in [0, 1]; the paper uses 0.8 */
  int32_t n_inner;            /* object/probe passes per iteration, >= 1         */
  int32_t probe_update_start; /* iterations before this index keep P fixed       */
  double denom_floor_rel;     /* delta = this * max(denominator), >= 0           */
  int32_t mem_kind;           /* DM_HOST or DM_DEVICE for dm_init's inputs       */
  dm_alloc_fn alloc;          /* NULL: cudaMallocAsync on the stream             */
  dm_free_fn free;
  void* alloc_user;
  void* stream;               /* cudaStream_t, or NULL for a library stream      */
                              /* (a blocking stream: ordered with the legacy     */
                              /* default stream; DM_DEVICE inputs written on     */
                              /* other streams must be complete at dm_init)      */
  int64_t scratch_bytes;      /* L2-resident Fourier-step scratch; 0 = 96 MiB.   */
                              /* Smaller values mean smaller view chunks.        */
  int32_t update_order;       /* DM_ORDER_GAUSS_SEIDEL (default) or DM_ORDER_JACOBI */
  int32_t psi_precision;      /* exit-wave storage: DM_PSI_FP32 (default) or      */
                              /* DM_PSI_FP16 (mixed-precision form, n = 64..256)  */
  double psi_switch;          /* DM_PSI_FP16 only: after the first iteration whose */
                              /* Eq. 6 object change is below this, the exit waves */
                              /* become complex64 (0 = never; see below)          */
} dm_params;

/* Exit-wave storage.  DM_PSI_FP32: complex64.  DM_PSI_FP16, the mixed-
 * precision form: the exit waves psi are stored as complex half (IEEE
 * binary16 real and imaginary parts, rounded to nearest even on every store)
 * and every operation on them is FP32, as in the FP32 form; the probe, the
 * object, the intensities, the Fourier scratch and all sums keep their
 * precision.  This halves the bytes of the three exit-wave passes of an
 * iteration (Fourier-step read and write, probe-update read).  Rounding psi
 * to 11 significant bits each iteration leaves an error floor near 1e-3
 * (relative, object), so with psi_switch > 0 dm_iterate returns to complex64
 * storage once the object's Eq. 6 change drops below psi_switch, and the
 * iteration is then the FP32 form.  The half form reads that monitor after
 * every iteration (one device-to-host copy and synchronisation each).  The
 * paper lists single precision as future work (Sec. V); this form goes one
 * step further for the stored exit waves only.  Not available with
 * dm_set_psi_error or in a dm_batch. */
#define DM_PSI_FP32 0
#define DM_PSI_FP16 1

/* Order of the overlap projection (Eqs. 4 and 5, written in the paper as
 * simultaneous updates).  Gauss-Seidel: the object from the probe the Fourier
 * step used, then each probe mode from the new object (n_inner passes).
 * Jacobi: both from the values the iteration started with, so each probe mode
 * divides by the old object; it requires n_inner = 1 (DM_EINVAL otherwise).
 * With view shards (dm_probe_partials) the Jacobi order uses the object that
 * was current before dm_object_apply. */
#define DM_ORDER_GAUSS_SEIDEL 0
#define DM_ORDER_JACOBI 1

/* Fill p with the defaults: beta 0.8, n_inner 1, probe_update_start 0,
 * denom_floor_rel 1e-6, mem_kind DM_HOST, no allocator, NULL stream,
 * default scratch, Gauss-Seidel order, complex64 exit waves; the sizes are
 * zeroed and must be set by the caller. */
void dm_params_default(dm_params* p);

/* Create a context on the current CUDA device: validate the parameters,
 * copy the positions, intensities, probe and object, and build the initial
 * exit waves psi_j^k = P_k O on every footprint (Sec. II, first step).
 * Returns DM_EINVAL for a bad size, a footprint outside the object, or an
 * intensity that is negative or not finite. On failure *out is NULL. */
int dm_init(dm_ctx** out, const dm_params* p, const int32_t* positions,
            const float* intensities, const float* probe0, const float* object0);

/* Enqueue n_iter >= 0 DM iterations (Eq. 3, then Eq. 5 and Eq. 4 n_inner
 * times, then Eq. 6).  Asynchronous with respect to the host. */
int dm_iterate(dm_ctx* ctx, int32_t n_iter);

/* Enqueue one piece of an iteration (DM_STEP_*).  DM_STEP_OBJECT and
 * DM_STEP_PROBE replace the current object / probe; no metric is written
 * and the iteration counter does not move.  DM_STEP_PROBE always divides by
 * the current object, whatever update_order says: the steps are the pieces
 * of a Gauss-Seidel iteration. */
int dm_run_step(dm_ctx* ctx, int32_t step);

/* Copy the current object [H][W][2], probe [M][N][N][2] or exit waves
 * [J][M][N][N][2] to `out` (host or device by mem_kind); synchronises. */
int dm_get_object(dm_ctx* ctx, float* out, int32_t mem_kind);
int dm_get_probe(dm_ctx* ctx, float* out, int32_t mem_kind);
int dm_get_exit_waves(dm_ctx* ctx, float* out, int32_t mem_kind);

/* Replace the exit waves, object or probe (resume from a checkpoint). */
int dm_set_exit_waves(dm_ctx* ctx, const float* in, int32_t mem_kind);
int dm_set_object(dm_ctx* ctx, const float* in, int32_t mem_kind);
int dm_set_probe(dm_ctx* ctx, const float* in, int32_t mem_kind);

/* Metrics of iteration `iter` (0-based; -1 = the last one).  eps_probe
 * receives M values.  Any output pointer may be NULL.  Only the last 1024
 * iterations are kept.  Synchronises; returns DM_ENONFINITE if any metric
 * computed so far was not finite. */
int dm_get_error(dm_ctx* ctx, int32_t iter, double* eps_obj, double* eps_probe,
                 double* fourier_err);

/* Exit-wave change eps_psi = sqrt(sum |psi' - psi|^2 / sum |psi'|^2) over
 * all views, modes and pixels of an iteration: the reading taken here of the
 * "psi error" that Sec. III counts among the costly steps without defining
 * it.  The Fourier step computes it only while tracking is on, because it
 * must read the old exit waves back (8 M N^2 more bytes per view and
 * iteration); it is off after dm_init.  dm_set_psi_error(ctx, 1) turns it on
 * (the first call allocates at most 256 bytes per view), 0 off; it
 * synchronises.
 * dm_get_psi_error reads iteration `iter` (0-based, -1 = the last; the last
 * 1024 are kept) into *eps_psi (host): NaN for an iteration that did not
 * track it (tracking off, a dm_batch iteration, or a sharded iteration);
 * synchronises. */
int dm_set_psi_error(dm_ctx* ctx, int32_t enable);
int dm_get_psi_error(dm_ctx* ctx, int32_t iter, double* eps_psi);

/* Diagnostic for the failure path: runs the library's two bounded device
 * waits on conditions that never become true (a counter spin-wait on a flag
 * nothing raises, an mbarrier wait on a phase nothing completes), on the
 * current device and its legacy default stream.  Each must give up after its
 * limit (1 s) and set the timeout status, which is what makes a stalled
 * Fourier step end with DM_ETIMEOUT instead of hanging.  Returns DM_OK when
 * both gave up and flagged it and the device still runs work afterwards,
 * DM_EINVAL if a wait did not give up as designed, DM_ECUDA on a CUDA error
 * (message in dm_last_error(NULL)).  *elapsed_ms (if non-NULL) receives the
 * device time of the test kernel (about 2000 ms).  Synchronises. */
int dm_selftest_bounded_waits(double* elapsed_ms);

/* FP32-pipe peak of the current device in TFLOP/s (a fused multiply-add
 * counted as two operations), measured by a kernel of eight independent FMA
 * chains per thread on four 512-thread CTAs per SM, timed with CUDA events
 * after a warm-up launch: the denominator of the arithmetic roofline of the
 * Fourier step's FP32 FFTs.  The paper has no counterpart; it is a
 * measurement utility.  Allocates 4 bytes of device memory, synchronises the
 * device.  Errors: DM_EINVAL (NULL), DM_ECUDA (message in dm_last_error(NULL)). */
int dm_fp32_peak(double* tflops);

/* Switch the exit-wave storage of a context (DM_PSI_FP32 or DM_PSI_FP16):
 * the exit waves are converted in place (rounded to complex half, or widened
 * exactly to complex64); captured graphs are dropped.  Synchronises.
 * dm_get_psi_precision reports the current storage and the iteration count
 * at which dm_iterate's automatic switch (psi_switch) returned to complex64
 * (-1 if it has not).  Errors: DM_EINVAL (unknown precision, n without a
 * half form, exit-wave change tracking on). */
int dm_set_psi_precision(dm_ctx* ctx, int32_t precision);
int dm_get_psi_precision(const dm_ctx* ctx, int32_t* precision, int64_t* switched_at);

/* Number of completed dm_iterate iterations. */
int64_t dm_iterations_done(const dm_ctx* ctx);

/* Power sum_u |P_k(u)|^2 of each probe mode (M doubles, host), the quantity
 * used to choose the number of modes (Sec. II).  Synchronises. */
int dm_get_mode_power(dm_ctx* ctx, double* out);

/* Wait for all enqueued work; report device-side errors. */
int dm_sync(dm_ctx* ctx);

/* Per-kernel-class timing with CUDA events on the context's stream.
 * dm_set_timing(ctx, 1) starts recording (and clears the totals);
 * dm_get_timing synchronises and returns the accumulated device time and
 * the number of launches of class `kernel` (DM_KERNEL_*). */
int dm_set_timing(dm_ctx* ctx, int32_t enable);
int dm_get_timing(dm_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches);
const char* dm_kernel_name(int32_t kernel);

/* Replay iterations as CUDA graphs (enable != 0) or launch every kernel
 * (0, the default).  With graphs on, dm_iterate captures one iteration per
 * pair of current object/probe buffers on first use (at most four graphs,
 * kept until dm_free) and replays it; the results are the same.  Iterations
 * with the probe frozen (probe_update_start) and iterations while timing is
 * on are launched kernel by kernel.  The first dm_iterate after enabling
 * performs the capture, so it must not itself run inside a stream capture. */
int dm_set_graph(dm_ctx* ctx, int32_t enable);

/* Choose the Fourier-step plan by measurement: every distinct combination
 * of scratch-ring size (48, 64, 96, 128, 160, 192 MiB), column-task size (64, 128,
 * 256 KiB of scratch) and strip buffers (2, 3) is timed on the first
 * sample_views views of the context (one warm-up and three timed runs of the
 * Fourier kernel each); where the scan has the split form (and the exit-wave
 * change is not tracked), that form is timed too at each ring size (48 to
 * 192 MiB), and so is the cluster form where the scan has it, so the choice
 * covers the form as well (dm_get_fourier_form reports it).  The fastest
 * form is kept for the whole scan, and so is the fastest plan of each form
 * (a batch or the exit-wave change runs the strip form with its best
 * plan whichever form won).  The exit
 * waves of the sample views are restored afterwards; the object sources are
 * recomputed by the next iteration, so results are unchanged.  Temporary
 * buffers (up to the largest ring plus a copy of the sample's exit waves)
 * come from the context's allocator.  *best_ms (if non-NULL) receives the
 * winning time per run on the sample.  Synchronises.  Errors: DM_EINVAL,
 * DM_ENOMEM, DM_ECUDA, DM_ETIMEOUT. */
int dm_autotune(dm_ctx* ctx, int32_t sample_views, double* best_ms);

/* The current Fourier-step plan: out[0] scratch-ring bytes, out[1] views per
 * chunk, out[2] strips per column task, out[3] strip buffers, out[4] CTAs.
 * For the split form out[2] is 0 and out[3] the item buffers of each of a
 * column task's two item lanes. */
int dm_get_plan(const dm_ctx* ctx, int64_t* out);

/* Three forms of the Fourier step (Eq. 3 with the constrained transform F_c
 * of Sec. II); all compute the same iteration to FP32 rounding.
 * DM_FOURIER_STRIP: row tasks take the row DFTs, column tasks the column
 * DFTs, the modulus projection and the inverse column DFTs of 2-column
 * strips of all modes; every frame size, mode count and exit-wave storage.
 * DM_FOURIER_SPLIT (256 x 256 frames with exactly 8 modes): the 256-point
 * column DFT is split into two radix-16 stages, the first in the row tasks
 * (over rows n1 + 16 n2 of one residue n1) and the second in the column
 * tasks, whose work items are 16 columns x 16 rows x 8 modes; the mode sum
 * of F_c is then a warp-shuffle reduction.  It keeps the intensities in a
 * second layout as well (4 N^2 bytes more per view).  The exit-wave change
 * (dm_set_psi_error) and dm_batch iterations run the strip form instead.  The split
 * form has a scratch ring of its own (160 MiB of 5 slots by default: more
 * views in flight let its tasks overlap more; dm_params.scratch_bytes, when
 * set, sizes both forms' rings).  Contexts that can run the split form start with it; dm_autotune
 * times both forms where both exist and keeps the faster, and
 * dm_set_fourier_form selects one explicitly
 * (DM_EINVAL for DM_FOURIER_SPLIT on other shapes); it synchronises and
 * drops captured iteration graphs.  dm_get_fourier_form
 * reports the form the next Fourier step runs.
 * DM_FOURIER_CLUSTER (64 x 64 or 128 x 128 frames with 1 to 8 modes): one thread-block
 * cluster per view and one CTA per mode; each CTA holds its mode's whole
 * frame in shared memory and runs both 1-D passes of both transforms there,
 * and the mode sums (S of the modulus projection, and c_j = sum_k conj(P_k)
 * psi'_k of Eq. 5) are reduce-scatters over the cluster's distributed shared
 * memory.  It has no scratch ring (dm_get_plan reports 0 bytes, 1 view per
 * cluster, 0 strips and buffers, and its CTAs).  Like the split form it
 * leaves the exit-wave change to the strip form; in a dm_batch a scan in the
 * cluster form keeps it (a launch of its own).  Contexts that have it start
 * in it with up to two modes at 128 x 128 and up to four at 64 x 64, and
 * with more when the scan has at most three views per cluster that fits the
 * GPU at once (the strip pipeline of such a short scan cannot fill);
 * dm_autotune times it against the strip plans where it exists. */
#define DM_FOURIER_STRIP 0
#define DM_FOURIER_SPLIT 1
#define DM_FOURIER_CLUSTER 2
int dm_set_fourier_form(dm_ctx* ctx, int32_t form);
int dm_get_fourier_form(const dm_ctx* ctx, int32_t* form);

/* Several scans advanced together (the batched form).  The contexts (same
 * device; any frame sizes, mode and view counts) keep their own data and
 * plans; an iteration of the batch runs, for each frame size, one persistent
 * Fourier-step launch over all scans of that size (up to 16 per launch; more
 * scans take further launches) in the strip form -- scans in the cluster form
 * take a cluster launch of their own instead -- then each scan's object and
 * probe updates and metrics.  Each scan's results equal those of dm_iterate
 * on it alone in the same form (the strip form for a scan whose own is the
 * split form).
 * The work runs on a stream the batch owns, ordered after the work queued on
 * every context's stream and before work queued on them afterwards.
 * dm_batch_set_graph(b, 1) captures a batch iteration as one CUDA graph per
 * combination of the scans' current buffers and replays it (iterations with
 * a frozen probe or with timing on are launched kernel by kernel).
 * The contexts must outlive the batch, and no other call may use them while
 * dm_batch_iterate runs.  Errors: DM_EINVAL, DM_ECUDA, DM_ENOMEM; the message
 * is in dm_batch_last_error (NULL: the last failed dm_batch_create). */
typedef struct dm_batch dm_batch;
int dm_batch_create(dm_batch** out, dm_ctx* const* ctxs, int32_t count);
int dm_batch_iterate(dm_batch* batch, int32_t n_iter);
int dm_batch_set_graph(dm_batch* batch, int32_t enable);
void dm_batch_free(dm_batch* batch);
const char* dm_batch_last_error(const dm_batch* batch);

/* Bytes of device memory the context holds. */
size_t dm_device_bytes(const dm_ctx* ctx);

/* Probe update (Eq. 4) for callers that cannot allocate device memory, such
 * as a host application that owns every byte of device memory and gives
 * this library no allocator, or code that must not call cudaMalloc/cudaFree.
 * The paper has no counterpart: this entry point exists only for those
 * callers.  It computes the same result as dm_run_step(DM_STEP_PROBE):
 *   probe_out_k(u) = sum_j conj(O(r_j+u)) psi_j^k(u) / (sum_j |O(r_j+u)|^2 + delta),
 *   delta = denom_floor_rel * max_u(denominator); pixels with a zero
 *   denominator keep probe_in.
 * All pointers are device pointers on the current device, laid out as for
 * dm_init (psi [J][M][N][N] complex, object [H][W] complex, positions
 * [J][2] int32, probes [M][N][N] complex); the caller owns them.
 * The call allocates nothing: its reduction scratch is one fixed 16 MiB
 * array inside the library (held by every GPU that loads the library until
 * the process exits), which bounds the size: about (24 M + 20) N^2 bytes
 * must fit in 16 MiB (N = 256 allows up to 9 modes).  Larger sizes return
 * DM_EINVAL.  The array's address on the current device is looked up on
 * every call.  All calls share the array: calls that overlap on the GPU
 * race, so order them on one stream.  The positions are checked on the
 * device before the update and a status word is read after it, so the call
 * synchronises `stream` and returns once probe_out holds the result; on a
 * stream that is being captured into a graph it returns DM_EINVAL and
 * enqueues nothing.  Errors: DM_EINVAL (sizes, NULL pointers, a footprint
 * outside the object, a capturing stream), DM_ETIMEOUT (a bounded device
 * wait of this call's update expired; probe_out is then not valid),
 * DM_ECUDA; the message is in dm_last_error(NULL). */
int dm_probe_update_static(const float* psi, const float* object, const int32_t* positions,
                           const float* probe_in, float* probe_out, int32_t n, int32_t modes,
                           int32_t views, int32_t obj_h, int32_t obj_w, double denom_floor_rel,
                           void* stream);

/* View-sharded overlap projection.  Sec. III spreads the views over GPUs:
 * every rank runs the Fourier step on its own views, and the sums of Eq. 5
 * and Eq. 4 over all views are formed by reducing per-rank partial sums
 * (MPI reduce + broadcast in the paper).  These calls expose that split for
 * a context that holds one shard of the views (same N, M, object size, beta
 * and denom_floor_rel on every shard; the views of the shards together are
 * the scan).  One iteration over S shard contexts, with "sum" any reduction
 * over the shards (host, NCCL, ...):
 *   for each shard: dm_run_step(DM_STEP_FOURIER)
 *   for each shard: dm_object_partials(num_s, den_s);  sum -> num, den
 *   for each shard: dm_object_apply(num, den)
 *   for each shard: dm_probe_partials(pnum_s, pden_s); sum -> pnum, pden
 *   for each shard: dm_probe_apply(pnum, pden)
 *   for each shard: dm_fourier_error_partials(e_s);    sum -> e
 *   for each shard: dm_finish_iteration(e)
 * which equals dm_iterate(1) on the unsharded scan with n_inner = 1 and the
 * probe updated (up to the order of the FP32 / FP64 sums).  Every shard ends
 * with the same object and probe; each keeps its own exit waves.
 *
 * dm_object_partials: numerator and denominator of Eq. 5 over this
 *   context's views, with the probe the Fourier step used:
 *   num [H][W] complex (float pairs) = sum_jk conj(P_k(r-r_j)) psi_j^k(r-r_j),
 *   summed in FP32 as the unsharded gather sums it;
 *   den [H][W] double = sum_jk |P_k(r-r_j)|^2 (0 where no view of the shard
 *   covers r), summed in FP32 over blocks of 32 views and in FP64 across
 *   blocks, returned without rounding to float.  Needs the Fourier step of
 *   this iteration to have run.
 * dm_object_apply: the object update from the sums over all shards, held
 *   in FP64: num [H][W][2] double, den [H][W] double.  O = num / (den +
 *   delta), delta = denom_floor_rel * max(den), formed in FP64 and rounded
 *   to float once; pixels with den = 0 keep their value.  It becomes the
 *   current object.
 * dm_probe_partials: numerator and denominator of Eq. 4 over this context's
 *   views with the current object, in FP64: num [M][N][N][2] double,
 *   den [N][N] double = sum_j |O(r_j+u)|^2.
 * dm_probe_apply: P_k = num_k / (den + delta), delta = denom_floor_rel *
 *   max(den); pixels with den = 0 keep their value.  It becomes the current
 *   probe.
 * dm_fourier_error_partials: sums[0] = sum_jq (sqrt S_j(q) - sqrt I_j(q))^2
 *   and sums[1] = sum_jq I_j(q) over this context's views, from its last
 *   Fourier step (host array of 2; synchronises).
 * dm_finish_iteration: records the iteration's metrics (Eq. 6 from the
 *   applied object and probe, E_F = sqrt(sums[0] / sums[1]) from the summed
 *   `sums`, a host array of 2) and counts the iteration.
 * num/den pointers follow mem_kind; the caller owns every buffer.  Errors:
 * DM_EINVAL (NULL pointers, bad mem_kind), DM_ECUDA. */
int dm_object_partials(dm_ctx* ctx, float* num, double* den, int32_t mem_kind);
int dm_object_apply(dm_ctx* ctx, const double* num, const double* den, int32_t mem_kind);
int dm_probe_partials(dm_ctx* ctx, double* num, double* den, int32_t mem_kind);
int dm_probe_apply(dm_ctx* ctx, const double* num, const double* den, int32_t mem_kind);
int dm_fourier_error_partials(dm_ctx* ctx, double* sums);
int dm_finish_iteration(dm_ctx* ctx, const double* sums);

/* Batched 2-D DFT of complex frames in two precision forms (the paper runs
 * FP64 and names single precision as future work, Sec. V).  N = 256 only.
 *   out[f][q] = sum_u in[f][u] exp(-+2 pi i (q . u) / N), unnormalised, '-'
 *   for the forward transform (inverse != 0 takes '+').
 * precision DM_DFT_FP32: the FP32 register radix-16 FFT of the Fourier step.
 * precision DM_DFT_BF16X3: each 16-point stage on the tensor cores as complex
 *   GEMMs with split BF16 operands (a = hi + lo, three products hi*hi +
 *   hi*lo + lo*hi per real GEMM) and FP32 accumulation (mma.sync); the
 *   twiddles between stages in FP32.
 * precision DM_DFT_BF16X3_TC05: each 256-point row transform as one dense
 *   complex GEMM (the row's 512 floats times the real-ified 512 x 512 DFT
 *   matrix) on the 5th-generation tensor cores (tcgen05.mma with its
 *   accumulators in tensor memory, the matrix streamed by TMA), with the same
 *   split BF16 operands and FP32 accumulation.  Each of its CTAs holds 512
 *   tensor-memory columns, so it runs one CTA per SM.
 * The two tensor-core forms' errors are bounded as stated in the tests
 * (relative L2 against an FP64 DFT).
 * in, work, out: device pointers on the current device, [frames][N][N]
 * complex (float pairs); work is caller-owned scratch of the same size and
 * must alias neither in nor out; out may equal in.  Work is enqueued on
 * `stream` (a cudaStream_t; NULL is the default stream).  The first call on a
 * device fills the library's twiddle tables: make it before any stream
 * capture.  Errors: DM_EINVAL, DM_ECUDA (message in dm_last_error(NULL)). */
#define DM_DFT_FP32 0
#define DM_DFT_BF16X3 1
#define DM_DFT_BF16X3_TC05 2
int dm_dft2(const float* in, float* work, float* out, int32_t n, int32_t frames, int32_t inverse,
            int32_t precision, void* stream);

/* Waits for the current device to finish its work, then reports whether a
 * bounded wait inside a DM_DFT_BF16X3_TC05 transform gave up (1 s; its
 * result is then not valid) since the last check: DM_ETIMEOUT, else DM_OK,
 * and clears the record.  DM_ECUDA on a CUDA error. */
int dm_dft2_check(void);

/* Learned warm start: a small convolutional encoder-decoder mapping one
 * recorded diffraction amplitude (128 x 128, float) to the object amplitude
 * and phase over the central 64 x 64 pixels of the view's footprint (2 x 64
 * x 64, float).  The paper has no network; it notes that the starting guess
 * may come from prior results (Sec. III).  Plain DM stays the judge of the
 * reconstruction that starts from the network's stitched prediction.
 * Six levels, 1,964,690 parameters: encoder 1->16->32->64->128->256->256
 * channels (3 x 3, stride 2, ReLU; 128 -> 2 pixels), decoder with nearest 2x
 * upsampling 256->256->128->64->32->16 (3 x 3, ReLU; 2 -> 64 pixels), head
 * 16->2 (3 x 3, linear).  Weights are BF16 in every product, with FP32
 * master copies, activations, gradients and accumulation; updates are Adam.
 * The loss (dm_net_set_loss) is the mean squared error over both output
 * channels (DM_NET_LOSS_MSE, the default) or the phase-gauge-invariant loss
 * (DM_NET_LOSS_GAUGE): one view's intensities do not change when its object
 * patch is multiplied by a constant phase factor, so each predicted complex
 * patch z = a exp(i phi) is compared with its target t after the best global
 * phase, (sum|z|^2 + sum|t|^2 - 2|sum conj(z) t|) per sample, averaged over
 * the batch's pixels.
 * Parameters are one flat FP32 array, per layer the weights [co][ci][3][3]
 * then the biases [co].  x, y and target are device pointers on the
 * network's device, [batch][1][128][128] and [batch][2][64][64]; grads and
 * params are host arrays of dm_net_param_count() floats; batch <=
 * max_batch.  dm_net_create draws He-normal weights from `seed`.
 * dm_net_gradients returns the loss gradients without updating;
 * dm_net_train_step applies one Adam step (learning rate lr) and, if `loss`
 * is not NULL, returns the batch loss.  The network allocates its own
 * buffers (cudaMallocAsync on a stream it owns).  That stream is a blocking
 * stream, so a call's work is ordered after work queued on the legacy
 * default stream; inputs produced on other streams must be complete before
 * the call.  Every call returns after its work is done, so the caller may
 * reuse x, target and y at once.  Errors: DM_EINVAL, DM_ENOMEM, DM_ECUDA
 * (message in dm_last_error(NULL)). */
typedef struct dm_net dm_net;
int dm_net_create(dm_net** out, int32_t max_batch, uint64_t seed);
int64_t dm_net_param_count(const dm_net* net);
int dm_net_get_params(dm_net* net, float* params);
int dm_net_set_params(dm_net* net, const float* params);
int dm_net_forward(dm_net* net, const float* x, int32_t batch, float* y);
int dm_net_gradients(dm_net* net, const float* x, const float* target, int32_t batch, float* grads,
                     double* loss);
int dm_net_train_step(dm_net* net, const float* x, const float* target, int32_t batch, float lr,
                      double* loss);
#define DM_NET_LOSS_MSE 0
#define DM_NET_LOSS_GAUGE 1
int dm_net_set_loss(dm_net* net, int32_t kind);
void dm_net_free(dm_net* net);

/* Release everything the context holds (NULL is ignored). */
void dm_free(dm_ctx* ctx);

/* Message of the last failure on ctx, or of the last failed dm_init when
 * ctx is NULL.  Valid until the next call on the same context. */
const char* dm_last_error(const dm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PTYCHO_DM_H */
