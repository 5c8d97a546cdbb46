// Internal interface between the host orchestrator (dm_api.cu) and the
// kernels (dm_fourier.cu, dm_overlap.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmk {

// Status bits the kernels OR into a device word; the host maps them to
// DM_E* codes at the next synchronising call.
enum : int {
  kStatusTimeout = 1,     // a bounded spin-wait expired
  kStatusNonFinite = 2,   // a metric was NaN or Inf
  kStatusBadInput = 4,    // an intensity was negative or not finite
};

constexpr int kThreads = 256;          // threads per CTA of every hot kernel
constexpr int kMetricsRing = 1024;     // iterations of metrics kept on the device
constexpr int kMaxModes = 16;
// One metrics row: eps_obj, fourier_err, eps_probe[kMaxModes], eps_psi.
constexpr int kRingRow = 3 + kMaxModes;
constexpr int kRingPsi = 2 + kMaxModes;
constexpr int kStripW = 2;             // columns per Fourier column strip
constexpr int kMaxStripBufs = 3;       // strip buffers of a column task
constexpr int kTwBytes = 2048;         // shared twiddle table (N <= 256 complex values)

// ---------------------------------------------------------------------------
// Fourier step (Eq. 3): one persistent launch over all views.
// Views are processed in chunks of B; each chunk goes through three task
// kinds that exchange data through an L2-resident scratch slot:
//   R: rows of (2 P O - psi) -> forward row DFT           -> slot  (T)
//   C: column strip, all modes -> forward column DFT, modulus projection,
//      inverse column DFT, U = beta T'' - T / N            -> slot  (U)
//   I: inverse row DFT of U, psi' = (2 - beta) P O + G[U], object source
//      c_j = sum_k conj(P_k) psi'_k                         -> psi, cview
// Task order is software-pipelined: stage s holds R(s), C(s - lag),
// I(s - 2 lag); a task waits (bounded) on counters of the chunk it depends on.
// ---------------------------------------------------------------------------
struct FourierArgs {
  int N, M, J, H, W;
  float beta;
  void* psi;              // [J][M][N][N] complex64, or complex half when psi16
  int psi16;              // 1: the exit waves are stored as complex half (mixed-precision form)
  const float* istrip;    // intensities in strip layout [J][NS][N][w]
  const float2* probe;    // [M][N][N]
  const float2* obj;      // [H][W]
  const int2* pos;        // [J] (row, col)
  float2* cview;          // [J][N][N] object source sum_k conj(P_k) psi_k
  float2* scratch;        // [nslot][B][M][N][N]
  double* ef_part;        // [J][CG] Fourier-error numerator partials
  double* psi_part;       // [J][RB][2] per I task: sum |psi' - psi|^2, sum |psi'|^2 (null: not
                          // tracked; the kernel instance must match, see launch_fourier)
  const float2* tw;       // twiddle tables (fourier_twiddles)
  int B, nchunks, lag, nslot;
  int RB;                 // row tasks per view (row blocks)
  int CG;                 // column tasks per view (strip groups)
  int SPG;                // strips per column task
  int w, lw;              // strip width (columns, = kStripW) and its log2
  int NS;                 // strips per view = N / w
  int strip_bufs;         // strip buffers of a column task (1 to kMaxStripBufs)
  int G;                  // strips a column task transforms at once (1 when the modes fill
                          // every slot): G * M slots busy out of kThreads / (w R2)
  int nstages, total_tasks;
  const int* stage_off;   // [nstages + 1] first task of each stage
  int* counters;          // [0] dispenser, then done R/C/I per view [J]
  int* status;
};

// The split-column form of the Fourier step (dm_fourier_split.cu) for N x N
// = 256 x 256 frames and 8 modes: the column DFT's first radix-16 stage runs
// in the row tasks, its second in the column tasks, whose items are 16
// columns x 16 rows x 8 modes (one TMA box of 128-byte rows).  Tasks per
// view: RB = CG = 16.  tmaps: [0] the scratch ring as rows of N complex
// values (box 16 x 128, 128-byte swizzle), [1] the intensities in the split
// layout (launch_intensity_split) as rows of 16 floats (box 16 x 16).
constexpr int kSplitN = 256;
constexpr int kSplitModes = 8;
constexpr int kSplitBufs = 3;          // item buffers per item lane of a column task
cudaError_t launch_fourier_split(const void* tmaps, const FourierArgs& a, int grid, size_t smem, cudaStream_t s);
size_t fourier_split_smem_bytes();
int fourier_split_occupancy(size_t smem);
// isplit[j][k1][x][k2] = inten[j][k1 + 16 k2][x] (J views of 256 x 256)
cudaError_t launch_intensity_split(float* isplit, const float* inten, int J, cudaStream_t s);

// The cluster form of the Fourier step (dm_fourier_cluster.cu) for 64 x 64
// and 128 x 128 frames and 1 to 8 modes: one thread-block cluster per view
// and one CTA per mode, each holding its mode's whole frame in shared memory;
// the mode sums are reduce-scatters over distributed shared memory.  It uses
// no scratch ring, counters or tensor maps; views go to clusters round-robin.
// It writes ef_part[j * M + mode] (M partials per view) and does not track
// the exit-wave change (psi_part).
constexpr int kClusterMaxModes = 8;
bool fourier_cluster_shape(int N, int M);   // whether the form exists for N x N frames and M modes
size_t fourier_cluster_smem_bytes(int N);
// clusters of M CTAs resident at once (0: the form cannot run); also sets the
// kernels' shared-memory limit, so it runs once before the first launch
int fourier_cluster_capacity(int N, int M);
cudaError_t launch_fourier_cluster(const FourierArgs& a, int nclusters, cudaStream_t s);

// Several scans of one frame size in one persistent Fourier launch: scan s
// owns tasks [base[s], base[s+1]) of the launch counter; its own plan,
// counters and scratch ring are in a[s], its scratch tensor map in map[s].
// The whole table is a kernel parameter (no tensor map in global memory).
constexpr int kMaxBatchScans = 16;
struct FourierBatch {
  CUtensorMap map[kMaxBatchScans];
  FourierArgs a[kMaxBatchScans];
  int base[kMaxBatchScans + 1];
  int nscan;
  int* dispenser;
};
cudaError_t launch_fourier_batch(const FourierBatch& b, int N, int grid, size_t smem, cudaStream_t s);
int fourier_batch_occupancy(int N, size_t smem);

// ---------------------------------------------------------------------------
// Object update (Eq. 5): gather over the views that cover each object tile.
// ---------------------------------------------------------------------------
constexpr int kObjTileH = 32, kObjTileW = 32;
constexpr int kObjBoxW = kObjTileW + 2;     // complex columns per TMA box
constexpr int kObjStages = 4;

struct ObjGatherArgs {
  int N, J, H, W, tiles_x;
  const int2* pos;
  const int* tile_ptr;     // [ntiles + 1]
  const int* tile_views;   // CSR lists (ascending view index)
  const float* p2;         // [N][N] sum_k |P_k|^2
  float2* num;             // [H][W]
  float* den;              // [H][W]
  double* den64;           // [H][W] the denominator before its float rounding (null: not written)
  unsigned* den_max_bits;  // max over the object (float bits, den >= 0)
  int* status;
};

struct ObjFinalArgs {
  int H, W;
  float delta_rel;
  const float2* num;
  const float* den;
  const unsigned* den_max_bits;
  const float2* o_start;   // object at the start of the iteration
  float2* o_new;
  double* part;            // [blocks][2]: sum |O_new - O_start|^2, sum |O_new|^2
};

// The object division from numerator and denominator sums held in FP64 (the
// view-sharded path, whose sums are added over shards in FP64): O = num /
// (den + delta) with delta = delta_rel * max(den), rounded to float once.
struct ObjFinal64Args {
  int H, W;
  double delta_rel;
  const double2* num;                  // [H][W]
  const double* den;                   // [H][W]
  const unsigned long long* den_max_bits;  // max of den (bits of the float-rounded value)
  const float2* o_start;
  float2* o_new;
  double* part;            // [blocks][2] as ObjFinalArgs
};
cudaError_t launch_obj_final64(const ObjFinal64Args& a, int blocks, cudaStream_t s);

// ---------------------------------------------------------------------------
// Probe update (Eq. 4): per-view-group partial sums, then a fixed-order
// FP64 reduction over the groups and the division.
// ---------------------------------------------------------------------------
constexpr int kProbePxPerThread = 2;   // pixels per thread for M <= 8 (1 above)
// depth of the views' shared-memory ring (2 CTAs per SM): complex64 exit
// waves 3 views, complex half (half the bytes per view) 5
template <class PsiT>
__host__ __device__ constexpr int probe_stages() { return sizeof(PsiT) == 8 ? 3 : 5; }

struct ProbePartialArgs {
  int N, M, J, H, W, groups;
  const void* psi;         // complex64, or complex half when psi16
  int psi16;
  const float2* obj;
  const int2* pos;
  float2* part_num;        // [groups][M][N*N]
  double* part_den;        // [groups][N*N]
  int* status;             // kStatusTimeout if a ring wait expired
};

struct ProbeFinalArgs {
  int N, M, groups;
  float delta_rel;
  const float2* part_num;
  const double* part_den;
  const float2* p_start;   // probe at the start of the iteration
  float2* p_new;
  float* p2;               // [N*N] sum_k |P_k|^2 of the new probe
  double* num_sum;         // [M][N*N][2] scratch for the FP64 sums
  double* den_sum;         // [N*N]
  unsigned long long* den_max_bits;
  double* part;            // [blocks][1 + 2M] partial Eq. 6 sums
};

// Launchers (return the launch error).
// tmaps: two CUtensorMap of the scratch ring (box of all modes, box of one mode)
cudaError_t launch_fourier(const void* tmaps, const FourierArgs& a, int grid, size_t smem, cudaStream_t s);
size_t fourier_smem_bytes(int N, int M, int bufs, int G);
int fourier_occupancy(int N, size_t smem);
int fourier_r2(int N);
// Twiddle tables of the Fourier kernel for frame size N (entries written to
// `tab` when non-null, double-precision angles); returns the entry count.
int fourier_twiddles(int N, float2* tab);

cudaError_t launch_obj_gather(const void* tmap, const ObjGatherArgs& a, int ntiles, cudaStream_t s);
cudaError_t launch_obj_final(const ObjFinalArgs& a, int blocks, cudaStream_t s);
cudaError_t launch_obj_source(float2* cview, const void* psi, int psi16, const float2* probe, int N, int M,
                              int J, cudaStream_t s);
// Pixels per probe tile and the probe-partial kernel's dynamic shared memory.
int probe_tile_px(int M);
size_t probe_partial_smem_bytes(int M);
// Probe partial sums; a persistent grid of min(items, 2 num_sms) CTAs (two per SM).
cudaError_t launch_probe_partial(const ProbePartialArgs& a, int num_sms, cudaStream_t s);
cudaError_t prepare_probe_partial(int M);
cudaError_t launch_probe_final(const ProbeFinalArgs& a, cudaStream_t s, int* blocks_out);
// The two halves of launch_probe_final: FP64 sums over the view groups (and
// max of the denominator), then the division and the Eq. 6 partials.
cudaError_t launch_probe_sum(const ProbeFinalArgs& a, cudaStream_t s);
cudaError_t launch_probe_div(const ProbeFinalArgs& a, cudaStream_t s, int* blocks_out);
// Maximum of a non-negative array as the bit pattern in *bits (start at 0);
// the f64 form records the float-rounded maximum.
cudaError_t launch_max_f32(const float* x, size_t n, unsigned* bits, cudaStream_t s);
cudaError_t launch_max_f64(const double* x, size_t n, unsigned long long* bits, cudaStream_t s);

cudaError_t launch_init_psi(void* psi, int psi16, const float2* probe, const float2* obj, const int2* pos,
                            int N, int M, int J, int W, cudaStream_t s);
// Exit waves between the two storage forms (n complex values): to_half = 1
// rounds complex64 to complex half, 0 widens complex half to complex64.
cudaError_t launch_psi_convert(void* dst, const void* src, size_t n, int to_half, cudaStream_t s);
// Whether the Fourier kernel has a complex-half form for N x N frames.
bool fourier_has_psi16(int N);
cudaError_t launch_intensity_layout(float* istrip, const float* inten, int N, int J, int w,
                                    double* isum_part, int* status, int* blocks_out, cudaStream_t s);
cudaError_t launch_p2(float* p2, const float2* probe, int N, int M, cudaStream_t s);
cudaError_t launch_reduce_sum(const double* in, long long n, int stride, int offset, double* out,
                              cudaStream_t s);
cudaError_t launch_metrics(const double* ef_part, long long n_ef, const double* isum,
                           const double* obj_part, int n_obj, const double* probe_part,
                           int n_probe, int M, int probe_updated, const double* psi_part, long long n_psi,
                           double* ring, long long* iter, int* status, cudaStream_t s);
cudaError_t launch_mode_power(const float2* probe, int N, int M, double* out, cudaStream_t s);
// flag: one zeroed int; status: two zeroed ints; ok: two ints (see k_wait_selftest)
cudaError_t launch_wait_selftest(const int* flag, int* status, int* ok, cudaStream_t s);

// Batched 2-D DFT of 256 x 256 frames (dm_dft.cu): tables and limits once
// per device, then the two row passes (precision 0 FP32, 1 split BF16 on the
// tensor cores).
cudaError_t prepare_dft256(cudaStream_t s);
cudaError_t launch_dft256(const float2* in, float2* work, float2* out, int frames, bool inverse, int precision,
                          cudaStream_t s);
// The tcgen05 form (dm_dft_tc.cu): its table, TMA view and shared-memory
// limit once per device, the two passes, and the status word of its bounded
// waits (synchronises the device, then reads and clears it).
cudaError_t prepare_dft256_tc05(cudaStream_t s);
cudaError_t launch_dft256_tc05(const float2* in, float2* work, float2* out, int frames, bool inverse,
                               cudaStream_t s);
cudaError_t dft256_tc05_status(int* timed_out);

// Message returned by dm_last_error(NULL) (calls made without a context).
void set_global_error(const char* msg);

}  // namespace dmk
