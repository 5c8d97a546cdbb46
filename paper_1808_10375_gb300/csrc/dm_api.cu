// Host side of the C ABI declared in include/dm.h: argument checking, device
// memory, the launch plans (Fourier task schedule, object-tile CSR lists, TMA
// tensor map, probe reduction groups) and the order of launches in one
// difference-map iteration (Sec. II: Eq. 3, then Eq. 5 and Eq. 4, then Eq. 6).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dm.h"
#include "dm_kernels.h"

namespace {

constexpr size_t kScratchBudget = 96ull << 20;   // L2-resident Fourier scratch
// The split form's default ring: its row and inverse row tasks wait at block
// barriers, and more views in flight give the SM other work meanwhile (at
// 256^2 x 8 modes: 5 slots of 8 views, 47.5 ms; 4 slots of 6 views, 53.5 ms).
constexpr size_t kSplitScratchBudget = 160ull << 20;
constexpr size_t kColumnSmemBudget = 100u << 10; // column strips in shared memory
constexpr size_t kColumnTaskBytes = 128u << 10;  // scratch bytes per column task
constexpr int kFourierLag = 1;                   // stages between task kinds

thread_local std::string g_init_error;

// The tunable parts of the Fourier-step plan.
struct FourierKnobs {
  size_t budget;      // scratch ring bytes (strip form)
  size_t task_bytes;  // scratch bytes per column task (sets the strips per task)
  int max_bufs;       // strip buffers of a column task, at most (1 to kMaxStripBufs)
  size_t split_budget;   // scratch ring bytes of the split form
};

struct TimedLaunch {
  int kind;
  cudaEvent_t start, stop;
};

}  // namespace

struct dm_ctx {
  uint32_t magic = 0x58434D44u;   // identifies a live context ('DMCX')
  dm_params p{};
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0;

  int N = 0, M = 0, J = 0, H = 0, W = 0;

  float2* psi = nullptr;         // exit waves, complex64 (also the staging buffer of the half form)
  void* psi16 = nullptr;         // exit waves as complex half (mixed-precision form), or null
  bool half = false;             // the exit waves currently live in psi16
  float2* probe[2] = {nullptr, nullptr};
  float2* obj[2] = {nullptr, nullptr};
  float2* cview = nullptr;
  float2* scratch = nullptr;
  float2* tw = nullptr;
  float2* num_O = nullptr;
  float2* part_num = nullptr;
  float* istrip = nullptr;
  float* p2 = nullptr;
  float* den_O = nullptr;
  double* den64_O = nullptr;    // [H][W] FP64 denominator (view shards; allocated on first use)
  double2* num64_O = nullptr;   // [H][W] summed FP64 numerator given to dm_object_apply
  unsigned long long* dmax64_O = nullptr;
  int2* pos = nullptr;
  int* counters = nullptr;
  int* stage_off = nullptr;
  int* status = nullptr;
  int* tile_ptr = nullptr;
  int* tile_views = nullptr;
  unsigned* dmax_O = nullptr;
  unsigned long long* dmax_P = nullptr;
  double* ef_part = nullptr;
  double* psi_part = nullptr;   // [J][RB][2] exit-wave change sums (allocated when tracking is on)
  bool psi_err = false;         // track the exit-wave change eps_psi
  double* isum_part = nullptr;
  double* isum = nullptr;
  double* obj_part = nullptr;
  double* probe_part = nullptr;
  double* part_den = nullptr;
  double* num_sum = nullptr;
  double* den_sum = nullptr;
  double* ring = nullptr;
  double* mode_pow = nullptr;
  double* ef_tot = nullptr;   // [2] summed Fourier-error terms of a sharded iteration
  long long* iter_dev = nullptr;   // iterations recorded (picks the metrics ring slot on the device)
  int cur_P = 0, cur_O = 0;

  dmk::FourierArgs fa{};
  FourierKnobs knobs{};
  int fgrid = 0;
  size_t fsmem = 0;
  size_t counters_bytes = 0;
  int tiles_x = 0, tiles_y = 0, obj_final_blocks = 0;
  CUtensorMap tmap_c;
  CUtensorMap tmap_s[2];   // scratch ring: box of all modes, box of one mode
  // the split-column form of the Fourier step (256 x 256 frames, 8 modes)
  bool split_ok = false;        // the form exists for this scan
  int form = DM_FOURIER_STRIP;  // the form dm_iterate runs
  float* isplit = nullptr;      // intensities in the split layout
  dmk::FourierArgs fs{};        // its plan (shares the scratch ring and counters of fa)
  int* stage_off_s = nullptr;
  int fsgrid = 0;
  size_t fssmem = 0;
  CUtensorMap tmap_split[2];    // scratch rows (box 16 x 128, swizzled), intensities (box 16 x 16)
  // the cluster form of the Fourier step (128 x 128 frames, 1 to 8 modes)
  bool cluster_ok = false;      // the form exists for this scan
  int ccap = 0;                 // clusters resident at once
  int ef_cg = 0;                // column tasks per view of the last Fourier launch (rows of ef_part)
  int probe_groups = 0;
  int probe_final_blocks = 0;
  int64_t iters = 0;
  int64_t switched_at = -1;      // iteration count when the exit waves went back to complex64
  bool use_graph = false;
  cudaStream_t cap_stream = nullptr;   // private stream the iteration graphs are captured on
  cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // by (cur_O, cur_P)

  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  double kms[DM_KERNEL_COUNT] = {};
  int64_t klaunch[DM_KERNEL_COUNT] = {};
};

namespace {

int fail(dm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_init_error = msg;
  return code;
}

int cuda_fail(dm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, DM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DM_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int dev_alloc(dm_ctx* c, void** out, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* ptr = nullptr;
  if (c->p.alloc) {
    ptr = c->p.alloc(bytes, c->p.alloc_user);
  } else if (cudaMallocAsync(&ptr, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (!ptr) return fail(c, DM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  c->allocs.emplace_back(ptr, bytes);
  c->bytes += bytes;
  *out = ptr;
  return DM_OK;
}

// Release one allocation of the context (nullptr is ignored).
void dev_free(dm_ctx* c, void* ptr) {
  if (!ptr) return;
  auto it = std::find_if(c->allocs.begin(), c->allocs.end(),
                         [&](const std::pair<void*, size_t>& a) { return a.first == ptr; });
  if (it == c->allocs.end()) return;
  if (c->p.alloc) c->p.free(it->first, c->p.alloc_user); else cudaFreeAsync(it->first, c->stream);
  c->bytes -= it->second;
  c->allocs.erase(it);
}

// The exit waves in their current storage form.
void* psi_cur(const dm_ctx* c) { return c->half ? c->psi16 : static_cast<void*>(c->psi); }
size_t psi_elem_bytes(const dm_ctx* c) { return c->half ? 4 : sizeof(float2); }

template <typename T>
int alloc_n(dm_ctx* c, T** out, size_t n) {
  return dev_alloc(c, reinterpret_cast<void**>(out), n * sizeof(T));
}

void release_all(dm_ctx* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& row : c->gexec)
    for (auto& g : row)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  if (c->cap_stream) { cudaStreamDestroy(c->cap_stream); c->cap_stream = nullptr; }
  for (auto& a : c->allocs) {
    if (c->p.alloc && c->p.free) c->p.free(a.first, c->p.alloc_user);
    else if (!c->p.alloc) cudaFreeAsync(a.first, c->stream);
  }
  c->allocs.clear();
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& t : c->pending) { cudaEventDestroy(t.start); cudaEventDestroy(t.stop); }
  c->pending.clear();
  for (auto e : c->event_pool) cudaEventDestroy(e);
  c->event_pool.clear();
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  c->stream = nullptr;
}

cudaEvent_t take_event(dm_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one launch with events when timing is on.
struct Timed {
  dm_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(dm_ctx* ctx, int k) : c(ctx), kind(k) {
    if (c->timing) {
      a = take_event(c);
      b = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~Timed() {
    if (c->timing && a && b) {
      cudaEventRecord(b, c->stream);
      c->pending.push_back({kind, a, b});
    }
  }
};

int collect_timing(dm_ctx* c) {
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  for (auto& t : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
      c->kms[t.kind] += ms;
      c->klaunch[t.kind] += 1;
    }
    c->event_pool.push_back(t.start);
    c->event_pool.push_back(t.stop);
  }
  c->pending.clear();
  return DM_OK;
}

int check_status(dm_ctx* c) {
  int st = 0;
  DM_CUDA(c, cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st & dmk::kStatusTimeout) return fail(c, DM_ETIMEOUT, "a bounded device-side wait expired");
  if (st & dmk::kStatusNonFinite) return fail(c, DM_ENONFINITE, "a metric was not finite");
  if (st & dmk::kStatusBadInput) return fail(c, DM_EINVAL, "an intensity was negative or not finite");
  return DM_OK;
}

int copy_in(dm_ctx* c, void* dst, const void* src, size_t bytes, int mem_kind) {
  DM_CUDA(c, cudaMemcpyAsync(dst, src, bytes, mem_kind == DM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                    : cudaMemcpyHostToDevice, c->stream));
  return DM_OK;
}

int copy_out(dm_ctx* c, void* dst, const void* src, size_t bytes, int mem_kind) {
  DM_CUDA(c, cudaMemcpyAsync(dst, src, bytes, mem_kind == DM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                    : cudaMemcpyDeviceToHost, c->stream));
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}

bool valid_n(int n) { return n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }

FourierKnobs default_knobs(const dm_ctx* c) {
  return {c->p.scratch_bytes > 0 ? (size_t)c->p.scratch_bytes : kScratchBudget, kColumnTaskBytes,
          dmk::kMaxStripBufs, c->p.scratch_bytes > 0 ? (size_t)c->p.scratch_bytes : kSplitScratchBudget};
}

// Host part of the plan for the first J views: the pipelined task order
// (stage offsets), the scratch ring, the strip buffers and the launch shape.
// Fills everything in `a` but the device pointers.
int fourier_schedule(dm_ctx* c, int J, const FourierKnobs& k, dmk::FourierArgs& a, std::vector<int>& off,
                     size_t& smem, int& grid, bool split = false) {
  const int N = c->N, M = c->M;
  const int R2 = dmk::fourier_r2(N);
  const int groups = dmk::kThreads / R2;
  const int GR = std::min(groups, N);
  a = dmk::FourierArgs{};
  a.N = N; a.M = M; a.J = J; a.H = c->H; a.W = c->W;
  a.RB = N / GR;
  a.w = dmk::kStripW;
  a.lw = 1;
  a.NS = N / a.w;
  const size_t strip_bytes = (size_t)M * N * a.w * sizeof(float2);
  int spg = 1;
  while (spg * 2 <= a.NS && strip_bytes * spg * 2 <= k.task_bytes) spg *= 2;
  a.SPG = spg;
  a.CG = a.NS / spg;
  // With fewer modes than column slots, G strips of the task are transformed
  // together so that G * M of the slots work (G divides SPG).
  a.G = 1;
  const int slots = dmk::kThreads / (a.w * R2);
  while (2 * a.G * M <= slots && 2 * a.G <= a.SPG) a.G *= 2;
  // Two or three strip buffers while two fit the shared-memory budget (a
  // third gives a strip and a half of prefetch unless it costs a resident
  // CTA, checked below), else one.
  a.strip_bufs =
      2 * a.G * (strip_bytes + (size_t)N * a.w * sizeof(float)) <= kColumnSmemBudget ? k.max_bufs : 1;
  a.strip_bufs = std::max(1, std::min(a.strip_bufs, dmk::kMaxStripBufs));
  if (split) {
    a.RB = dmk::kSplitN / 16;
    a.CG = dmk::kSplitN / 16;
    a.SPG = 0;
    a.G = 1;
    a.strip_bufs = 0;
  }
  a.lag = kFourierLag;
  // Slots: R(s), C(s - lag) and I(s - 2 lag) use 2 lag + 1 of them; each
  // further slot lets the row tasks run a chunk further ahead of the inverse
  // row tasks that free their slot.  The split form's row and inverse row
  // tasks wait at block barriers and gain from that slack (256^2 x 8 modes, 8
  // views per chunk: 4 slots 50.1 ms, 5 slots 47.5 ms); the strip form does not.
  a.nslot = 2 * a.lag + (split ? 3 : 2);
  const size_t view_bytes = (size_t)M * N * N * sizeof(float2);
  size_t B = (split ? k.split_budget : k.budget) / ((size_t)a.nslot * view_bytes);
  B = std::max<size_t>(1, std::min<size_t>(B, (size_t)J));
  a.B = (int)B;
  a.nchunks = (J + a.B - 1) / a.B;
  a.nstages = a.nchunks + 2 * a.lag;
  off.assign(a.nstages + 1, 0);
  auto nv = [&](int ch) { return std::min(a.B, J - ch * a.B); };
  long long total = 0;
  for (int s = 0; s < a.nstages; ++s) {
    off[s] = (int)total;
    if (s < a.nchunks) total += (long long)nv(s) * a.RB;
    if (s - a.lag >= 0 && s - a.lag < a.nchunks) total += (long long)nv(s - a.lag) * a.CG;
    if (s - 2 * a.lag >= 0 && s - 2 * a.lag < a.nchunks) total += (long long)nv(s - 2 * a.lag) * a.RB;
  }
  off[a.nstages] = (int)total;
  if (total >= (1ll << 31)) return fail(c, DM_EINVAL, "too many Fourier tasks");
  a.total_tasks = (int)total;
  a.beta = c->p.beta;
  if (split) {
    // the split form: 16 row tasks (one per row residue n1), 16 column tasks
    // (one per k1) and 16 inverse row tasks per view; no strips
    smem = dmk::fourier_split_smem_bytes();
    const int occ = dmk::fourier_split_occupancy(smem);
    if (occ < 1) return fail(c, DM_ECUDA, "split Fourier kernel does not fit on an SM");
    grid = std::max(1, std::min(a.total_tasks, occ * c->num_sms));
    return DM_OK;
  }
  // an extra strip buffer is only worth it while it costs no resident CTA
  while (a.strip_bufs > 1 &&
         dmk::fourier_occupancy(N, dmk::fourier_smem_bytes(N, M, a.strip_bufs, a.G)) <
             dmk::fourier_occupancy(N, dmk::fourier_smem_bytes(N, M, a.strip_bufs - 1, a.G)))
    --a.strip_bufs;
  smem = dmk::fourier_smem_bytes(N, M, a.strip_bufs, a.G);
  const int occ = dmk::fourier_occupancy(N, smem);   // also sets the kernel's shared-memory limit
  if (occ < 1) return fail(c, DM_ECUDA, "Fourier kernel does not fit on an SM");
  grid = std::max(1, std::min(a.total_tasks, occ * c->num_sms));
  return DM_OK;
}

// TMA views of a scratch ring for the column tasks: planes of N x N complex
// values (8-byte elements), one plane per (view, mode).  map[0]'s box is
// kStripW columns x N rows x M modes (strip loads), map[1]'s the same with
// one mode (the per-mode stores of U).
int encode_scratch_map(dm_ctx* c, const dmk::FourierArgs& a, float2* scratch, CUtensorMap* map) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  DM_CUDA(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess) return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const int N = a.N, M = a.M;
  const cuuint64_t e = sizeof(float2);
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)a.nslot * a.B * M};
  const cuuint64_t strides[2] = {(cuuint64_t)N * e, (cuuint64_t)N * N * e};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int i = 0; i < 2; ++i) {
    const cuuint32_t box[3] = {(cuuint32_t)a.w, (cuuint32_t)N, (cuuint32_t)(i == 0 ? M : 1)};
    const CUresult r = encode(map + i, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, scratch, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled (scratch) failed (" + std::to_string((int)r) + ")");
  }
  return DM_OK;
}

size_t scratch_elems(const dmk::FourierArgs& a) { return (size_t)a.nslot * a.B * a.M * a.N * a.N; }

// TMA views of the split form: the scratch ring as rows of N complex values
// (one row per (view, k1, n1, mode)), box 16 columns x 16 M rows with the
// 128-byte swizzle; the split-layout intensities as rows of 16 floats (one
// row per (view, k1, column)), box 16 x 16.
int encode_split_maps(dm_ctx* c, const dmk::FourierArgs& a, float2* scratch, CUtensorMap* map) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  DM_CUDA(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess) return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const int N = a.N, M = a.M;
  const cuuint32_t estr[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)a.nslot * a.B * 16 * 16 * M};
    const cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float2)};
    const cuuint32_t box[2] = {16, (cuuint32_t)(16 * M)};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, scratch, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled (split scratch) failed (" + std::to_string((int)r) + ")");
  }
  {
    const cuuint64_t dims[2] = {16, (cuuint64_t)c->J * 16 * N};
    const cuuint64_t strides[1] = {16 * sizeof(float)};
    const cuuint32_t box[2] = {16, 16};
    const CUresult r = encode(map + 1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->isplit, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled (split intensities) failed (" + std::to_string((int)r) + ")");
  }
  return DM_OK;
}

// Whether the next Fourier step runs the split form (the exit-wave change is
// tracked by the strip form only).
bool use_split(const dm_ctx* c) { return c->split_ok && c->form == DM_FOURIER_SPLIT && !c->psi_err; }
bool use_cluster(const dm_ctx* c) { return c->cluster_ok && c->form == DM_FOURIER_CLUSTER && !c->psi_err; }

// Plan the Fourier step of the whole scan with knobs `k` and allocate its
// buffers (scratch ring, stage offsets, counters, Fourier-error partials).
int plan_fourier(dm_ctx* c, const FourierKnobs& k) {
  dmk::FourierArgs& a = c->fa;
  std::vector<int> off;
  int rc;
  if ((rc = fourier_schedule(c, c->J, k, a, off, c->fsmem, c->fgrid))) return rc;
  // the split form has a ring of its own size (split_budget) in the same buffer
  std::vector<int> soff;
  if (c->split_ok && (rc = fourier_schedule(c, c->J, k, c->fs, soff, c->fssmem, c->fsgrid, true))) return rc;
  if ((rc = alloc_n(c, &c->scratch, std::max(scratch_elems(a), c->split_ok ? scratch_elems(c->fs) : 0)))) return rc;
  if ((rc = alloc_n(c, &c->stage_off, off.size()))) return rc;
  // completed tasks are counted per view
  c->counters_bytes = sizeof(int) * (1 + 3 * (size_t)c->J);
  if ((rc = dev_alloc(c, reinterpret_cast<void**>(&c->counters), c->counters_bytes))) return rc;
  if ((rc = alloc_n(c, &c->ef_part, (size_t)c->J * std::max(a.CG, dmk::kSplitN / 16)))) return rc;
  DM_CUDA(c, cudaMemcpyAsync(c->stage_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice,
                             c->stream));
  DM_CUDA(c, cudaStreamSynchronize(c->stream));  // `off` is a host temporary
  if ((rc = encode_scratch_map(c, a, c->scratch, c->tmap_s))) return rc;
  if (c->split_ok) {
    dmk::FourierArgs& s = c->fs;
    if ((rc = alloc_n(c, &c->stage_off_s, soff.size()))) return rc;
    DM_CUDA(c, cudaMemcpyAsync(c->stage_off_s, soff.data(), soff.size() * sizeof(int), cudaMemcpyHostToDevice,
                               c->stream));
    DM_CUDA(c, cudaStreamSynchronize(c->stream));
    if ((rc = encode_split_maps(c, s, c->scratch, c->tmap_split))) return rc;
    s.psi = psi_cur(c); s.psi16 = c->half ? 1 : 0;
    s.istrip = c->isplit; s.pos = c->pos; s.cview = c->cview;
    s.scratch = c->scratch; s.ef_part = c->ef_part; s.tw = c->tw;
    s.stage_off = c->stage_off_s; s.counters = c->counters; s.status = c->status;
    s.psi_part = nullptr;
  }
  a.psi = psi_cur(c); a.psi16 = c->half ? 1 : 0;
  a.istrip = c->istrip; a.pos = c->pos; a.cview = c->cview;
  a.scratch = c->scratch; a.ef_part = c->ef_part; a.tw = c->tw;
  a.stage_off = c->stage_off; a.counters = c->counters; a.status = c->status;
  a.psi_part = c->psi_err ? c->psi_part : nullptr;
  c->knobs = k;
  return DM_OK;
}

int plan_fourier(dm_ctx* c) { return plan_fourier(c, default_knobs(c)); }

int plan_object(dm_ctx* c, const std::vector<int32_t>& hpos) {
  const int N = c->N, J = c->J;
  c->tiles_x = (c->W + dmk::kObjTileW - 1) / dmk::kObjTileW;
  c->tiles_y = (c->H + dmk::kObjTileH - 1) / dmk::kObjTileH;
  const int ntiles = c->tiles_x * c->tiles_y;
  std::vector<int> cnt(ntiles + 1, 0);
  for (int j = 0; j < J; ++j) {
    const int r = hpos[2 * j], q = hpos[2 * j + 1];
    for (int ty = r / dmk::kObjTileH; ty <= (r + N - 1) / dmk::kObjTileH; ++ty)
      for (int tx = q / dmk::kObjTileW; tx <= (q + N - 1) / dmk::kObjTileW; ++tx) cnt[ty * c->tiles_x + tx + 1]++;
  }
  for (int t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
  std::vector<int> fill(cnt.begin(), cnt.end() - 1), views(cnt[ntiles]);
  for (int j = 0; j < J; ++j) {
    const int r = hpos[2 * j], q = hpos[2 * j + 1];
    for (int ty = r / dmk::kObjTileH; ty <= (r + N - 1) / dmk::kObjTileH; ++ty)
      for (int tx = q / dmk::kObjTileW; tx <= (q + N - 1) / dmk::kObjTileW; ++tx)
        views[fill[ty * c->tiles_x + tx]++] = j;
  }
  int rc;
  if ((rc = alloc_n(c, &c->tile_ptr, cnt.size()))) return rc;
  if ((rc = alloc_n(c, &c->tile_views, std::max<size_t>(1, views.size())))) return rc;
  DM_CUDA(c, cudaMemcpyAsync(c->tile_ptr, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  if (!views.empty())
    DM_CUDA(c, cudaMemcpyAsync(c->tile_views, views.data(), views.size() * sizeof(int), cudaMemcpyHostToDevice,
                               c->stream));
  DM_CUDA(c, cudaStreamSynchronize(c->stream));

  // TMA view of the object sources: a 2-D array of floats, 2N wide, J*N rows.
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  DM_CUDA(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess) return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)J * N};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * N) * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * dmk::kObjBoxW), (cuuint32_t)dmk::kObjTileH};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&c->tmap_c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->cview, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, DM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  c->obj_final_blocks = 2 * c->num_sms;
  if ((rc = alloc_n(c, &c->num_O, (size_t)c->H * c->W))) return rc;
  if ((rc = alloc_n(c, &c->den_O, (size_t)c->H * c->W))) return rc;
  if ((rc = alloc_n(c, &c->dmax_O, 1))) return rc;
  if ((rc = alloc_n(c, &c->obj_part, 2 * (size_t)c->obj_final_blocks))) return rc;
  return DM_OK;
}

int plan_probe(dm_ctx* c) {
  DM_CUDA(c, dmk::prepare_probe_partial(c->M));
  const int nn = c->N * c->N;
  const int tp = dmk::probe_tile_px(c->M);
  const int tiles = (nn + tp - 1) / tp;
  // view groups such that tiles x groups work items are a multiple of the SM
  // count (the probe-partial grid has two persistent CTAs per SM)
  int g = c->num_sms / std::gcd(tiles, c->num_sms);
  g = std::max(1, std::min(g, c->J));
  c->probe_groups = g;
  c->probe_final_blocks = std::max(1, std::min((nn + dmk::kThreads - 1) / dmk::kThreads, 256));
  int rc;
  if ((rc = alloc_n(c, &c->part_num, (size_t)g * c->M * nn))) return rc;
  if ((rc = alloc_n(c, &c->part_den, (size_t)g * nn))) return rc;
  if ((rc = alloc_n(c, &c->num_sum, 2 * (size_t)c->M * nn))) return rc;
  if ((rc = alloc_n(c, &c->den_sum, (size_t)nn))) return rc;
  if ((rc = alloc_n(c, &c->dmax_P, 1))) return rc;
  if ((rc = alloc_n(c, &c->probe_part, (size_t)c->probe_final_blocks * 2 * c->M))) return rc;
  return DM_OK;
}

int run_fourier(dm_ctx* c) {
  DM_CUDA(c, cudaMemsetAsync(c->counters, 0, c->counters_bytes, c->stream));
  const bool split = use_split(c);
  dmk::FourierArgs& a = split ? c->fs : c->fa;
  a.probe = c->probe[c->cur_P];
  a.obj = c->obj[c->cur_O];
  a.psi = psi_cur(c);
  a.psi16 = c->half ? 1 : 0;
  if (use_cluster(c)) {
    c->ef_cg = c->M;   // one Fourier-error partial per view and mode
    Timed t(c, DM_KERNEL_FOURIER);
    DM_CUDA(c, dmk::launch_fourier_cluster(a, std::min(c->J, c->ccap), c->stream));
    return DM_OK;
  }
  c->ef_cg = a.CG;
  Timed t(c, DM_KERNEL_FOURIER);
  if (split) DM_CUDA(c, dmk::launch_fourier_split(c->tmap_split, a, c->fsgrid, c->fssmem, c->stream));
  else DM_CUDA(c, dmk::launch_fourier(c->tmap_s, a, c->fgrid, c->fsmem, c->stream));
  return DM_OK;
}

// Eq. 5, part 1: numerator and denominator over the context's views from
// the current object sources (num_O, den_O, and the maximum of den_O).
int run_object_gather(dm_ctx* c, double* den64 = nullptr) {
  DM_CUDA(c, cudaMemsetAsync(c->dmax_O, 0, sizeof(unsigned), c->stream));
  dmk::ObjGatherArgs g{};
  g.N = c->N; g.J = c->J; g.H = c->H; g.W = c->W; g.tiles_x = c->tiles_x;
  g.pos = c->pos; g.tile_ptr = c->tile_ptr; g.tile_views = c->tile_views; g.p2 = c->p2;
  g.num = c->num_O; g.den = c->den_O; g.den64 = den64; g.den_max_bits = c->dmax_O; g.status = c->status;
  Timed t(c, DM_KERNEL_OBJECT_GATHER);
  DM_CUDA(c, dmk::launch_obj_gather(&c->tmap_c, g, c->tiles_x * c->tiles_y, c->stream));
  return DM_OK;
}

// Eq. 5, part 2: obj[nxt] = num_O / (den_O + delta); o_start = obj[cur].
int run_object_final(dm_ctx* c) {
  dmk::ObjFinalArgs f{};
  f.H = c->H; f.W = c->W; f.delta_rel = (float)c->p.denom_floor_rel;
  f.num = c->num_O; f.den = c->den_O; f.den_max_bits = c->dmax_O;
  f.o_start = c->obj[c->cur_O]; f.o_new = c->obj[c->cur_O ^ 1]; f.part = c->obj_part;
  Timed t(c, DM_KERNEL_OBJECT_FINAL);
  DM_CUDA(c, dmk::launch_obj_final(f, c->obj_final_blocks, c->stream));
  return DM_OK;
}

// Eq. 5 into obj[nxt] from the current object sources; o_start = obj[cur].
int run_object(dm_ctx* c) {
  int rc;
  if ((rc = run_object_gather(c))) return rc;
  return run_object_final(c);
}

dmk::ProbeFinalArgs probe_final_args(dm_ctx* c) {
  dmk::ProbeFinalArgs f{};
  f.N = c->N; f.M = c->M; f.groups = c->probe_groups; f.delta_rel = (float)c->p.denom_floor_rel;
  f.part_num = c->part_num; f.part_den = c->part_den; f.p_start = c->probe[c->cur_P];
  f.p_new = c->probe[c->cur_P ^ 1]; f.p2 = c->p2; f.num_sum = c->num_sum; f.den_sum = c->den_sum;
  f.den_max_bits = c->dmax_P; f.part = c->probe_part;
  return f;
}

// Eq. 4, part 1: per-group partial sums from psi and object `o`, then their
// FP64 sums over the groups (num_sum, den_sum and the maximum of den_sum).
int run_probe_sums(dm_ctx* c, const float2* o) {
  dmk::ProbePartialArgs a{};
  a.N = c->N; a.M = c->M; a.J = c->J; a.H = c->H; a.W = c->W; a.groups = c->probe_groups;
  a.psi = psi_cur(c); a.psi16 = c->half ? 1 : 0;
  a.obj = o; a.pos = c->pos; a.part_num = c->part_num; a.part_den = c->part_den;
  a.status = c->status;
  {
    Timed t(c, DM_KERNEL_PROBE_PARTIAL);
    DM_CUDA(c, dmk::launch_probe_partial(a, c->num_sms, c->stream));
  }
  DM_CUDA(c, cudaMemsetAsync(c->dmax_P, 0, sizeof(unsigned long long), c->stream));
  Timed t(c, DM_KERNEL_PROBE_FINAL);
  DM_CUDA(c, dmk::launch_probe_sum(probe_final_args(c), c->stream));
  return DM_OK;
}

// Eq. 4, part 2: probe[nxt] = num_sum / (den_sum + delta); p_start = probe[cur].
int run_probe_div(dm_ctx* c) {
  int blocks = 0;
  Timed t(c, DM_KERNEL_PROBE_FINAL);
  DM_CUDA(c, dmk::launch_probe_div(probe_final_args(c), c->stream, &blocks));
  return DM_OK;
}

// Eq. 4 into probe[nxt] from psi and object `o`; p_start = probe[cur].
int run_probe(dm_ctx* c, const float2* o) {
  int rc;
  if ((rc = run_probe_sums(c, o))) return rc;
  return run_probe_div(c);
}

// Eq. 6 and the Fourier error into the metrics ring; `psi` when this
// iteration's Fourier step wrote the exit-wave change sums.
int run_metrics(dm_ctx* c, const double* ef, long long n_ef, const double* isum, bool upd, bool psi) {
  Timed t(c, DM_KERNEL_METRICS);
  const bool track = psi && c->fa.psi_part;
  DM_CUDA(c, dmk::launch_metrics(ef, n_ef, isum, c->obj_part, c->obj_final_blocks, c->probe_part,
                                 c->probe_final_blocks, c->M, upd ? 1 : 0, track ? c->fa.psi_part : nullptr,
                                 track ? (long long)c->J * c->fa.RB : 0, c->ring, c->iter_dev, c->status,
                                 c->stream));
  return DM_OK;
}

int check_ctx(dm_ctx* c) {
  if (!c || c->magic != 0x58434D44u) return DM_EINVAL;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return DM_OK;
}

}  // namespace

namespace dmk {
void set_global_error(const char* msg) { g_init_error = msg ? msg : ""; }
}  // namespace dmk

extern "C" {

void dm_params_default(dm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->beta = 0.8f;
  p->n_inner = 1;
  p->probe_update_start = 0;
  p->denom_floor_rel = 1e-6;
  p->mem_kind = DM_HOST;
  p->psi_precision = DM_PSI_FP32;
  p->psi_switch = 0.0;
}

int dm_init(dm_ctx** out, const dm_params* p, const int32_t* positions, const float* intensities,
            const float* probe0, const float* object0) {
  g_init_error.clear();
  if (!out) return fail(nullptr, DM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, DM_EINVAL, "params is NULL");
  if (!positions || !intensities || !probe0 || !object0) return fail(nullptr, DM_EINVAL, "an input pointer is NULL");
  if (!valid_n(p->n)) return fail(nullptr, DM_EINVAL, "n must be 16, 32, 64, 128 or 256");
  if (p->modes < 1 || p->modes > dmk::kMaxModes) return fail(nullptr, DM_EINVAL, "modes must be in 1..16");
  if (p->views < 1 || (long long)p->views * p->n >= (1ll << 31))
    return fail(nullptr, DM_EINVAL, "views out of range");
  if (p->obj_h < p->n || p->obj_w < p->n || (long long)p->obj_h * p->obj_w >= (1ll << 31))
    return fail(nullptr, DM_EINVAL, "object must be at least n x n and below 2^31 pixels");
  if (!(p->beta >= 0.f && p->beta <= 1.f)) return fail(nullptr, DM_EINVAL, "beta must be in [0, 1]");
  if (p->n_inner < 1) return fail(nullptr, DM_EINVAL, "n_inner must be >= 1");
  if (p->probe_update_start < 0) return fail(nullptr, DM_EINVAL, "probe_update_start must be >= 0");
  if (!(p->denom_floor_rel >= 0.0) || !std::isfinite(p->denom_floor_rel))
    return fail(nullptr, DM_EINVAL, "denom_floor_rel must be finite and >= 0");
  if (p->mem_kind != DM_HOST && p->mem_kind != DM_DEVICE) return fail(nullptr, DM_EINVAL, "bad mem_kind");
  if ((p->alloc == nullptr) != (p->free == nullptr)) return fail(nullptr, DM_EINVAL, "alloc and free go together");
  if (p->scratch_bytes < 0) return fail(nullptr, DM_EINVAL, "scratch_bytes must be >= 0");
  if (p->update_order != DM_ORDER_GAUSS_SEIDEL && p->update_order != DM_ORDER_JACOBI)
    return fail(nullptr, DM_EINVAL, "unknown update_order");
  if (p->update_order == DM_ORDER_JACOBI && p->n_inner != 1)
    return fail(nullptr, DM_EINVAL, "the Jacobi order takes n_inner = 1");
  if (p->psi_precision != DM_PSI_FP32 && p->psi_precision != DM_PSI_FP16)
    return fail(nullptr, DM_EINVAL, "unknown psi_precision");
  if (p->psi_precision == DM_PSI_FP16 && !dmk::fourier_has_psi16(p->n))
    return fail(nullptr, DM_EINVAL, "complex-half exit waves need n = 64, 128 or 256");
  if (!(p->psi_switch >= 0.0) || !std::isfinite(p->psi_switch))
    return fail(nullptr, DM_EINVAL, "psi_switch must be finite and >= 0");
  if (p->mem_kind == DM_HOST) {
    for (int j = 0; j < p->views; ++j) {
      const int r = positions[2 * j], q = positions[2 * j + 1];
      if (r < 0 || q < 0 || r > p->obj_h - p->n || q > p->obj_w - p->n)
        return fail(nullptr, DM_EINVAL, "footprint of view " + std::to_string(j) + " lies outside the object");
    }
  }

  dm_ctx* c = new (std::nothrow) dm_ctx();
  if (!c) return fail(nullptr, DM_ENOMEM, "out of host memory");
  c->p = *p;
  c->N = p->n; c->M = p->modes; c->J = p->views; c->H = p->obj_h; c->W = p->obj_w;
  auto bail = [&](int rc) {
    g_init_error = c->err.empty() ? g_init_error : c->err;
    release_all(c);
    delete c;
    return rc;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { cuda_fail(c, e, "cudaGetDevice"); return bail(DM_ECUDA); }
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) { cuda_fail(c, e, "cudaDeviceGetAttribute"); return bail(DM_ECUDA); }
  if (p->stream) {
    c->stream = static_cast<cudaStream_t>(p->stream);
  } else {
    // a blocking stream, ordered with work on the legacy default stream
    // (where device inputs are usually produced)
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault);
    if (e != cudaSuccess) { cuda_fail(c, e, "cudaStreamCreate"); return bail(DM_ECUDA); }
    c->own_stream = true;
  }

  const int N = c->N, M = c->M, J = c->J;
  const size_t nn = (size_t)N * N;
  // positions: validate on the host (they also drive the object tiling)
  std::vector<int32_t> hpos(2 * (size_t)J);
  if (p->mem_kind == DM_DEVICE) {
    e = cudaMemcpy(hpos.data(), positions, hpos.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { cuda_fail(c, e, "copy positions"); return bail(DM_ECUDA); }
  } else {
    std::memcpy(hpos.data(), positions, hpos.size() * sizeof(int32_t));
  }
  for (int j = 0; j < J; ++j) {
    const int r = hpos[2 * j], q = hpos[2 * j + 1];
    if (r < 0 || q < 0 || r > c->H - N || q > c->W - N) {
      fail(c, DM_EINVAL, "footprint of view " + std::to_string(j) + " lies outside the object");
      return bail(DM_EINVAL);
    }
  }

  int rc;
#define DM_TRY(x) do { if ((rc = (x)) != DM_OK) return bail(rc); } while (0)
  DM_TRY(alloc_n(c, &c->psi, (size_t)J * M * nn));
  if (p->psi_precision == DM_PSI_FP16) {
    DM_TRY(dev_alloc(c, &c->psi16, (size_t)J * M * nn * 4));
    c->half = true;
  }
  DM_TRY(alloc_n(c, &c->cview, (size_t)J * nn));
  DM_TRY(alloc_n(c, &c->istrip, (size_t)J * nn));
  c->split_ok = N == dmk::kSplitN && M == dmk::kSplitModes;
  // the split form where it exists (faster on the 10,000-view 8-mode workload
  // with its own ring size); dm_autotune may pick the other
  c->form = c->split_ok ? DM_FOURIER_SPLIT : DM_FOURIER_STRIP;
  if (c->split_ok) DM_TRY(alloc_n(c, &c->isplit, (size_t)J * nn));
  if (dmk::fourier_cluster_shape(N, M)) {
    c->ccap = dmk::fourier_cluster_capacity(N, M);
    c->cluster_ok = c->ccap > 0;
    // the cluster form for up to two modes at 128 x 128 and up to four at
    // 64 x 64, and for scans of at most three views per resident cluster
    // (Fourier step, ms, strip against cluster, at 2,500 views: 128 x 128
    // with 1 mode 1.02 / 0.54, 2 modes 1.06 / 0.98, 3 modes 1.50 / 1.65,
    // 4 modes 1.77 / 2.07 (0.109 / 0.096 at 108 views, even at 144); 64 x 64
    // with 1 mode 0.215 / 0.113, 4 modes 0.476 / 0.447, 8 modes 0.862 /
    // 1.007 (0.074 / 0.046 at 100 views))
    const int any_length = N == 64 ? 4 : 2;
    if (c->cluster_ok && (M <= any_length || J <= 3 * c->ccap)) c->form = DM_FOURIER_CLUSTER;
  }
  DM_TRY(alloc_n(c, &c->probe[0], (size_t)M * nn));
  DM_TRY(alloc_n(c, &c->probe[1], (size_t)M * nn));
  DM_TRY(alloc_n(c, &c->obj[0], (size_t)c->H * c->W));
  DM_TRY(alloc_n(c, &c->obj[1], (size_t)c->H * c->W));
  DM_TRY(alloc_n(c, &c->p2, nn));
  DM_TRY(alloc_n(c, &c->pos, (size_t)J));
  const int ntw = dmk::fourier_twiddles(N, nullptr);
  DM_TRY(alloc_n(c, &c->tw, (size_t)ntw));
  DM_TRY(alloc_n(c, &c->status, 1));
  DM_TRY(alloc_n(c, &c->isum, 1));
  DM_TRY(alloc_n(c, &c->ring, (size_t)dmk::kMetricsRing * dmk::kRingRow));
  DM_TRY(alloc_n(c, &c->mode_pow, (size_t)M));
  DM_TRY(alloc_n(c, &c->ef_tot, 2));
  DM_TRY(alloc_n(c, &c->iter_dev, 1));
  if ((e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream)) != cudaSuccess) { cuda_fail(c, e, "memset"); return bail(DM_ECUDA); }
  if ((e = cudaMemsetAsync(c->iter_dev, 0, sizeof(long long), c->stream)) != cudaSuccess) { cuda_fail(c, e, "memset"); return bail(DM_ECUDA); }
  if ((e = cudaMemsetAsync(c->ring, 0, sizeof(double) * dmk::kMetricsRing * dmk::kRingRow, c->stream)) != cudaSuccess) {
    cuda_fail(c, e, "memset"); return bail(DM_ECUDA);
  }

  std::vector<float2> htw(ntw);
  dmk::fourier_twiddles(N, htw.data());
  DM_TRY(copy_in(c, c->tw, htw.data(), ntw * sizeof(float2), DM_HOST));
  DM_TRY(copy_in(c, c->pos, hpos.data(), hpos.size() * sizeof(int32_t), DM_HOST));
  DM_TRY(copy_in(c, c->probe[0], probe0, (size_t)M * nn * sizeof(float2), p->mem_kind));
  DM_TRY(copy_in(c, c->obj[0], object0, (size_t)c->H * c->W * sizeof(float2), p->mem_kind));

  DM_TRY(plan_fourier(c));
  DM_TRY(plan_object(c, hpos));
  DM_TRY(plan_probe(c));

  // intensities: strip layout for the column tasks, checked, and sum_q I
  const float* dev_i = intensities;
  float* tmp = nullptr;
  if (p->mem_kind == DM_HOST) {
    DM_TRY(alloc_n(c, &tmp, (size_t)J * nn));
    DM_TRY(copy_in(c, tmp, intensities, (size_t)J * nn * sizeof(float), DM_HOST));
    dev_i = tmp;
  }
  double* isum_part = nullptr;
  DM_TRY(alloc_n(c, &isum_part, 2048));
  int ib = 0;
  if ((e = dmk::launch_intensity_layout(c->istrip, dev_i, N, J, c->fa.w, isum_part, c->status, &ib, c->stream)) !=
      cudaSuccess) { cuda_fail(c, e, "intensity layout"); return bail(DM_ECUDA); }
  if ((e = dmk::launch_reduce_sum(isum_part, ib, 1, 0, c->isum, c->stream)) != cudaSuccess) {
    cuda_fail(c, e, "intensity sum"); return bail(DM_ECUDA);
  }
  if (c->split_ok && (e = dmk::launch_intensity_split(c->isplit, dev_i, J, c->stream)) != cudaSuccess) {
    cuda_fail(c, e, "split intensity layout"); return bail(DM_ECUDA);
  }
  if ((e = dmk::launch_p2(c->p2, c->probe[0], N, M, c->stream)) != cudaSuccess) { cuda_fail(c, e, "p2"); return bail(DM_ECUDA); }
  if ((e = dmk::launch_init_psi(psi_cur(c), c->half ? 1 : 0, c->probe[0], c->obj[0], c->pos, N, M, J, c->W,
                                c->stream)) != cudaSuccess) {
    cuda_fail(c, e, "initial exit waves"); return bail(DM_ECUDA);
  }
  DM_TRY(check_status(c));
  // the staging buffers are no longer needed
  for (void* t : {static_cast<void*>(tmp), static_cast<void*>(isum_part)}) {
    if (!t) continue;
    auto it = std::find_if(c->allocs.begin(), c->allocs.end(), [&](const std::pair<void*, size_t>& a) { return a.first == t; });
    if (it != c->allocs.end()) {
      if (c->p.alloc) c->p.free(it->first, c->p.alloc_user); else cudaFreeAsync(it->first, c->stream);
      c->bytes -= it->second;
      c->allocs.erase(it);
    }
  }
#undef DM_TRY
  *out = c;
  return DM_OK;
}

}  // extern "C"

namespace {

// The object Eq. 4 divides by within an iteration, after the object update
// wrote obj[cur_O ^ 1]: the new object (Gauss-Seidel) or the old one (Jacobi).
const float2* probe_object(const dm_ctx* c) {
  return c->obj[c->p.update_order == DM_ORDER_JACOBI ? c->cur_O : c->cur_O ^ 1];
}

// Every launch of one iteration (Eq. 3, then Eq. 5 and Eq. 4 n_inner times,
// then Eq. 6), enqueued on the context's stream; no host state changes.
int enqueue_iteration(dm_ctx* c, bool upd) {
  int rc;
  if ((rc = run_fourier(c))) return rc;
  for (int pass = 0; pass < c->p.n_inner; ++pass) {
    if (pass > 0) {
      Timed t(c, DM_KERNEL_OTHER);
      DM_CUDA(c, dmk::launch_obj_source(c->cview, psi_cur(c), c->half ? 1 : 0, c->probe[c->cur_P ^ 1], c->N, c->M, c->J,
                                             c->stream));
    }
    if ((rc = run_object(c))) return rc;
    if (!upd) break;  // later passes would repeat the same object update
    if ((rc = run_probe(c, probe_object(c)))) return rc;
  }
  return run_metrics(c, c->ef_part, (long long)c->J * c->ef_cg, c->isum, upd, true);
}

// The iteration for the current (object, probe) buffers as an instantiated
// CUDA graph, captured on first use.
int iteration_graph(dm_ctx* c, cudaGraphExec_t* out) {
  cudaGraphExec_t& g = c->gexec[c->cur_O][c->cur_P];
  if (!g) {
    // Capture on a private stream (the context's stream may be the legacy
    // default stream, which cannot be captured); the graph is then launched
    // on the context's stream.
    if (!c->cap_stream) DM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    DM_CUDA(c, cudaStreamSynchronize(c->stream));   // the graph must not overtake queued work
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    cudaError_t e0 = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e0 != cudaSuccess) { c->stream = user; return cuda_fail(c, e0, "cudaStreamBeginCapture"); }
    const int rc = enqueue_iteration(c, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->stream = user;
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    const cudaError_t e2 = cudaGraphInstantiate(&g, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) { g = nullptr; return cuda_fail(c, e2, "cudaGraphInstantiate"); }
  }
  *out = g;
  return DM_OK;
}

// Switch the exit-wave storage between complex64 and complex half.
int set_psi_precision(dm_ctx* c, int32_t precision) {
  const bool want_half = precision == DM_PSI_FP16;
  if (want_half == c->half) return DM_OK;
  const size_t n = (size_t)c->J * c->M * c->N * c->N;
  if (want_half) {
    if (!dmk::fourier_has_psi16(c->N)) return fail(c, DM_EINVAL, "complex-half exit waves need n = 64, 128 or 256");
    if (c->psi_err) return fail(c, DM_EINVAL, "the exit-wave change is tracked with complex64 exit waves only");
    int rc;
    if (!c->psi16 && (rc = dev_alloc(c, &c->psi16, n * 4))) return rc;
    DM_CUDA(c, dmk::launch_psi_convert(c->psi16, c->psi, n, 1, c->stream));
  } else {
    DM_CUDA(c, dmk::launch_psi_convert(c->psi, c->psi16, n, 0, c->stream));
  }
  c->half = want_half;
  c->switched_at = want_half ? -1 : c->iters;
  // captured iterations launched the other kernel instances on the other buffer
  for (auto& row : c->gexec)
    for (auto& g : row)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return DM_OK;
}

}  // namespace

extern "C" {

int dm_iterate(dm_ctx* c, int32_t n_iter) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_iter < 0) return fail(c, DM_EINVAL, "n_iter must be >= 0");
  for (int it = 0; it < n_iter; ++it) {
    const bool upd = c->iters >= c->p.probe_update_start;
    if (c->use_graph && upd && !c->timing) {
      cudaGraphExec_t g = nullptr;
      if ((rc = iteration_graph(c, &g))) return rc;
      DM_CUDA(c, cudaGraphLaunch(g, c->stream));
    } else if ((rc = enqueue_iteration(c, upd))) {
      return rc;
    }
    c->cur_O ^= 1;
    if (upd) c->cur_P ^= 1;
    c->iters++;
    // mixed-precision form: complex-half exit waves until the object's Eq. 6
    // change falls below psi_switch, then complex64 for the rest of the run
    if (c->half && c->p.psi_switch > 0.0) {
      double eps_obj = 0.0;
      DM_CUDA(c, cudaMemcpyAsync(&eps_obj, c->ring + (size_t)((c->iters - 1) % dmk::kMetricsRing) * dmk::kRingRow,
                                 sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      DM_CUDA(c, cudaStreamSynchronize(c->stream));
      if (eps_obj < c->p.psi_switch && (rc = set_psi_precision(c, DM_PSI_FP32))) return rc;
    }
  }
  return DM_OK;
}

int dm_set_psi_precision(dm_ctx* c, int32_t precision) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (precision != DM_PSI_FP32 && precision != DM_PSI_FP16) return fail(c, DM_EINVAL, "unknown psi precision");
  DM_CUDA(c, cudaStreamSynchronize(c->stream));   // no captured iteration is in flight
  if ((rc = set_psi_precision(c, precision))) return rc;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}

int dm_get_psi_precision(const dm_ctx* c, int32_t* precision, int64_t* switched_at) {
  if (!c || c->magic != 0x58434D44u) return DM_EINVAL;
  if (precision) *precision = c->half ? DM_PSI_FP16 : DM_PSI_FP32;
  if (switched_at) *switched_at = c->switched_at;
  return DM_OK;
}

int dm_autotune(dm_ctx* c, int32_t sample_views, double* best_ms) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (sample_views < 1) return fail(c, DM_EINVAL, "sample_views must be >= 1");
  const int Js = std::min<int>(sample_views, c->J);
  const int N = c->N;
  struct Plan {
    FourierKnobs k;
    dmk::FourierArgs a;
    std::vector<int> off;
    size_t smem;
    int grid;
    bool split;
    bool cluster = false;
  };
  std::vector<Plan> plans;
  size_t max_scr = 0, max_off = 0, max_cnt = 0;
  // the split form (where the scan has it, and unless the exit-wave change
  // is tracked) competes with the strip plans; its only knob is the ring
  for (int split = 0; split <= (c->split_ok && !c->psi_err ? 1 : 0); ++split)
    for (size_t mb : {48, 64, 96, 128, 160, 192})
      for (size_t kb : {64, 128, 256})
        for (int b : {2, 3}) {
          Plan pl;
          // a plan of one form carries the current ring size of the other
          pl.k = split ? FourierKnobs{c->knobs.budget, c->knobs.task_bytes, c->knobs.max_bufs, mb << 20}
                       : FourierKnobs{mb << 20, kb << 10, b, c->knobs.split_budget};
          pl.split = split != 0;
          if ((rc = fourier_schedule(c, Js, pl.k, pl.a, pl.off, pl.smem, pl.grid, pl.split))) return rc;
          bool dup = false;
          for (const Plan& q : plans)
            dup = dup || (q.split == pl.split && q.a.B == pl.a.B && q.a.SPG == pl.a.SPG &&
                          q.a.strip_bufs == pl.a.strip_bufs);
          if (dup) continue;
          max_scr = std::max(max_scr, scratch_elems(pl.a));
          max_off = std::max(max_off, pl.off.size());
          max_cnt = std::max(max_cnt, 1 + 3 * (size_t)Js);
          plans.push_back(std::move(pl));
        }
  // the cluster form (no knobs) where the scan has it
  if (c->cluster_ok && !c->psi_err) {
    Plan pl;
    pl.k = c->knobs;
    pl.a = c->fa;
    pl.a.J = Js;
    pl.smem = 0;
    pl.grid = std::min(Js, c->ccap);
    pl.split = false;
    pl.cluster = true;
    plans.push_back(std::move(pl));
  }
  float2 *scr = nullptr, *psi_save = nullptr;
  int *offd = nullptr, *cnt = nullptr;
  double* ef = nullptr;
  const size_t psi_elems = (size_t)Js * c->M * N * N;
  auto release = [&]() {
    cudaStreamSynchronize(c->stream);
    for (void* q : {(void*)scr, (void*)psi_save, (void*)offd, (void*)cnt, (void*)ef}) dev_free(c, q);
  };
  if ((rc = alloc_n(c, &scr, max_scr)) || (rc = alloc_n(c, &psi_save, psi_elems)) ||
      (rc = alloc_n(c, &offd, max_off)) || (rc = alloc_n(c, &cnt, max_cnt)) ||
      (rc = alloc_n(c, &ef, (size_t)Js * (N / dmk::kStripW)))) {
    release();
    return rc;
  }
  // the tuning runs change the exit waves of the sample views: keep a copy
  DM_CUDA(c, cudaMemcpyAsync(psi_save, psi_cur(c), psi_elems * psi_elem_bytes(c), cudaMemcpyDeviceToDevice,
                             c->stream));
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  double best = 1e300;
  FourierKnobs best_k = c->knobs;
  bool best_split = use_split(c), best_cluster = use_cluster(c);
  // the best plan of each form is kept as well: batches and the exit-wave
  // change run the strip form whichever form wins
  double best_strip_t = 1e300, best_split_t = 1e300;
  FourierKnobs strip_k = c->knobs;
  size_t split_budget = c->knobs.split_budget;
  constexpr int kReps = 3;
  for (Plan& pl : plans) {
    dmk::FourierArgs a = pl.a;
    a.psi = psi_cur(c); a.psi16 = c->half ? 1 : 0;
    a.istrip = pl.split ? c->isplit : c->istrip; a.pos = c->pos; a.cview = c->cview; a.scratch = scr; a.ef_part = ef;
    a.tw = c->tw; a.stage_off = offd; a.counters = cnt; a.status = c->status;
    a.probe = c->probe[c->cur_P]; a.obj = c->obj[c->cur_O];
    CUtensorMap map[2];
    if (!pl.cluster && (rc = pl.split ? encode_split_maps(c, a, scr, map) : encode_scratch_map(c, a, scr, map))) {
      release();
      return rc;
    }
    cudaError_t e = cudaSuccess;
    if (!pl.cluster) {
      e = cudaMemcpyAsync(offd, pl.off.data(), pl.off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      // sets the kernel's shared-memory limit for this plan
      if (pl.split) dmk::fourier_split_occupancy(pl.smem); else dmk::fourier_occupancy(N, pl.smem);
    }
    for (int r = 0; r <= kReps && e == cudaSuccess; ++r) {   // the first run warms up
      if (r == 1) e = cudaEventRecord(e0, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * (1 + 3 * (size_t)Js), c->stream);
      if (e == cudaSuccess)
        e = pl.cluster ? dmk::launch_fourier_cluster(a, pl.grid, c->stream)
            : pl.split ? dmk::launch_fourier_split(map, a, pl.grid, pl.smem, c->stream)
                       : dmk::launch_fourier(map, a, pl.grid, pl.smem, c->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { release(); return cuda_fail(c, e, "autotune run"); }
    const double t = ms / kReps;
    if (!pl.split && !pl.cluster && t < best_strip_t) { best_strip_t = t; strip_k = pl.k; }
    if (pl.split && t < best_split_t) { best_split_t = t; split_budget = pl.k.split_budget; }
    if (t < best) {
      best = t;
      best_split = pl.split;
      best_cluster = pl.cluster;
    }
  }
  c->event_pool.push_back(e0);
  c->event_pool.push_back(e1);
  DM_CUDA(c, cudaMemcpyAsync(psi_cur(c), psi_save, psi_elems * psi_elem_bytes(c), cudaMemcpyDeviceToDevice,
                             c->stream));
  release();
  if ((rc = check_status(c))) return rc;
  // re-plan the whole scan with the fastest knobs (captured graphs hold the
  // old plan's arguments)
  for (auto& row : c->gexec)
    for (auto& g : row)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  for (void* q : {(void*)c->scratch, (void*)c->stage_off, (void*)c->counters, (void*)c->ef_part, (void*)c->stage_off_s})
    dev_free(c, q);
  c->scratch = nullptr; c->stage_off = nullptr; c->counters = nullptr; c->ef_part = nullptr; c->stage_off_s = nullptr;
  best_k = strip_k;
  best_k.split_budget = split_budget;
  if ((rc = plan_fourier(c, best_k))) return rc;
  c->form = best_cluster ? DM_FOURIER_CLUSTER : best_split ? DM_FOURIER_SPLIT : DM_FOURIER_STRIP;
  if (best_ms) *best_ms = best;
  return DM_OK;
}

int dm_get_plan(const dm_ctx* c, int64_t* out) {
  if (!c || !out) return DM_EINVAL;
  if (use_cluster(c)) {   // no scratch ring: one view per cluster of M CTAs at a time
    out[0] = 0;
    out[1] = 1;
    out[2] = 0;
    out[3] = 0;
    out[4] = (int64_t)std::min(c->J, c->ccap) * c->M;
    return DM_OK;
  }
  const bool split = use_split(c);
  const dmk::FourierArgs& a = split ? c->fs : c->fa;
  out[0] = (int64_t)scratch_elems(a) * (int64_t)sizeof(float2);
  out[1] = a.B;
  out[2] = split ? 0 : c->fa.SPG;
  out[3] = split ? dmk::kSplitBufs : c->fa.strip_bufs;
  out[4] = split ? c->fsgrid : c->fgrid;
  return DM_OK;
}

int dm_set_fourier_form(dm_ctx* c, int32_t form) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (form != DM_FOURIER_STRIP && form != DM_FOURIER_SPLIT && form != DM_FOURIER_CLUSTER)
    return fail(c, DM_EINVAL, "unknown Fourier form");
  if (form == DM_FOURIER_SPLIT && !c->split_ok)
    return fail(c, DM_EINVAL, "the split form needs 256 x 256 frames and 8 modes");
  if (form == DM_FOURIER_CLUSTER && !c->cluster_ok)
    return fail(c, DM_EINVAL, "the cluster form needs 64 x 64 or 128 x 128 frames and 1 to 8 modes");
  if (form == c->form) return DM_OK;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));   // no captured iteration is in flight below
  c->form = form;
  // captured iterations hold the previous Fourier-step instance
  for (auto& row : c->gexec)
    for (auto& g : row)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return DM_OK;
}

int dm_get_fourier_form(const dm_ctx* c, int32_t* form) {
  if (!c || c->magic != 0x58434D44u || !form) return DM_EINVAL;
  *form = use_cluster(c) ? DM_FOURIER_CLUSTER : use_split(c) ? DM_FOURIER_SPLIT : DM_FOURIER_STRIP;
  return DM_OK;
}

}  // extern "C"

// A batch of contexts advanced together: per frame size, one persistent
// Fourier launch over all its scans (at most kMaxBatchScans per launch),
// then each scan's overlap projection and metrics, all on the batch's
// stream.
struct dm_batch {
  std::vector<dm_ctx*> ctx;
  struct Group {
    int N = 0;
    std::vector<int> scans;
    size_t smem = 0;
    int grid = 0;
  };
  std::vector<Group> groups;
  int device = 0;
  cudaStream_t stream = nullptr;
  int* dispensers = nullptr;   // one per group
  cudaEvent_t ev = nullptr;
  // the scans' overlap projections run concurrently, one stream per scan,
  // forked after the Fourier launches and joined before the iteration ends
  std::vector<cudaStream_t> lanes;
  cudaEvent_t begin = nullptr;   // start of an iteration: the cluster-form scans' lanes fork here
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  bool use_graph = false;
  std::vector<std::pair<std::vector<int>, cudaGraphExec_t>> graphs;   // by the scans' buffer parities
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

int batch_fail(dm_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg; else g_batch_error = msg;
  return code;
}

#define DM_BCUDA(b, call)                                                               \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return batch_fail(b, DM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Every launch of one batch iteration on the batch's stream.
int enqueue_batch_iteration(dm_batch* b) {
  DM_BCUDA(b, cudaEventRecord(b->begin, b->stream));
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    auto& g = b->groups[gi];
    dmk::FourierBatch fb{};
    fb.dispenser = b->dispensers + gi;
    int base = 0, ns = 0;
    for (int scan : g.scans) {
      dm_ctx* c = b->ctx[scan];
      c->fa.probe = c->probe[c->cur_P];
      c->fa.obj = c->obj[c->cur_O];
      c->fa.psi = psi_cur(c);
      c->fa.psi16 = c->half ? 1 : 0;
      if (use_cluster(c)) {
        // a scan in the cluster form keeps it: a launch of its own on the
        // scan's lane, concurrent with the other scans' launches (its overlap
        // projections follow on the same lane)
        c->ef_cg = c->M;
        DM_BCUDA(b, cudaStreamWaitEvent(b->lanes[scan], b->begin, 0));
        DM_BCUDA(b, dmk::launch_fourier_cluster(c->fa, std::min(c->J, c->ccap), b->lanes[scan]));
        continue;
      }
      fb.a[ns] = c->fa;
      fb.map[ns] = c->tmap_s[0];
      c->ef_cg = c->fa.CG;   // the persistent launch runs the strip form
      fb.base[ns] = base;
      base += c->fa.total_tasks;
      DM_BCUDA(b, cudaMemsetAsync(c->counters, 0, c->counters_bytes, b->stream));
      ++ns;
    }
    if (ns == 0) continue;
    fb.nscan = ns;
    fb.base[ns] = base;
    DM_BCUDA(b, cudaMemsetAsync(fb.dispenser, 0, sizeof(int), b->stream));
    DM_BCUDA(b, dmk::launch_fourier_batch(fb, g.N, g.grid, g.smem, b->stream));
  }
  DM_BCUDA(b, cudaEventRecord(b->fork, b->stream));
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    dm_ctx* c = b->ctx[i];
    const bool upd = c->iters >= c->p.probe_update_start;
    cudaStream_t own = c->stream;
    // the strip-form scans follow the persistent launches
    if (!use_cluster(c)) DM_BCUDA(b, cudaStreamWaitEvent(b->lanes[i], b->fork, 0));
    c->stream = b->lanes[i];
    int rc = DM_OK;
    for (int pass = 0; pass < c->p.n_inner && rc == DM_OK; ++pass) {
      if (pass > 0) {
        const cudaError_t e = dmk::launch_obj_source(c->cview, psi_cur(c), c->half ? 1 : 0, c->probe[c->cur_P ^ 1], c->N, c->M, c->J,
                                                     c->stream);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "object source");
      }
      if (rc == DM_OK) rc = run_object(c);
      if (!upd) break;
      if (rc == DM_OK) rc = run_probe(c, probe_object(c));
    }
    if (rc == DM_OK) rc = run_metrics(c, c->ef_part, (long long)c->J * c->ef_cg, c->isum, upd, false);
    c->stream = own;
    if (rc) return batch_fail(b, rc, c->err);
    DM_BCUDA(b, cudaEventRecord(b->joins[i], b->lanes[i]));
    DM_BCUDA(b, cudaStreamWaitEvent(b->stream, b->joins[i], 0));
  }
  return DM_OK;
}

}  // namespace

extern "C" {

int dm_batch_create(dm_batch** out, dm_ctx* const* ctxs, int32_t count) {
  g_batch_error.clear();
  if (!out) return batch_fail(nullptr, DM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || count < 1) return batch_fail(nullptr, DM_EINVAL, "no contexts");
  auto* b = new dm_batch();
  b->device = ctxs[0]->device;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) { delete b; return batch_fail(nullptr, DM_EINVAL, "a context is NULL"); }
    if (ctxs[i]->device != b->device) { delete b; return batch_fail(nullptr, DM_EINVAL, "contexts on different devices"); }
    if (ctxs[i]->half) { delete b; return batch_fail(nullptr, DM_EINVAL, "a context stores complex-half exit waves"); }
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) { delete b; return batch_fail(nullptr, DM_EINVAL, "a context appears twice"); }
    b->ctx.push_back(ctxs[i]);
  }
  cudaSetDevice(b->device);
  for (int i = 0; i < count; ++i) {
    const int N = b->ctx[i]->N;
    dm_batch::Group* g = nullptr;
    for (auto& q : b->groups)
      if (q.N == N && (int)q.scans.size() < dmk::kMaxBatchScans) g = &q;
    if (!g) { b->groups.emplace_back(); g = &b->groups.back(); g->N = N; }
    g->scans.push_back(i);
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  for (auto& g : b->groups) {
    long long tasks = 0;
    for (int s : g.scans) {
      g.smem = std::max(g.smem, b->ctx[s]->fsmem);
      tasks += b->ctx[s]->fa.total_tasks;
    }
    const int occ = dmk::fourier_batch_occupancy(g.N, g.smem);
    if (occ < 1) { delete b; return batch_fail(nullptr, DM_ECUDA, "batched Fourier kernel does not fit on an SM"); }
    g.grid = (int)std::max<long long>(1, std::min<long long>(tasks, (long long)occ * sms));
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->begin, cudaEventDisableTiming);
  b->lanes.assign(b->ctx.size(), nullptr);
  b->joins.assign(b->ctx.size(), nullptr);
  for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->lanes[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&b->dispensers), sizeof(int) * b->groups.size(), b->stream);
  if (e != cudaSuccess) {
    dm_batch_free(b);
    return batch_fail(nullptr, DM_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  *out = b;
  return DM_OK;
}

int dm_batch_iterate(dm_batch* b, int32_t n_iter) {
  if (!b) return DM_EINVAL;
  if (n_iter < 0) return batch_fail(b, DM_EINVAL, "n_iter must be >= 0");
  DM_BCUDA(b, cudaSetDevice(b->device));
  // the batch's stream follows the work queued on every context's stream
  for (dm_ctx* c : b->ctx) {
    DM_BCUDA(b, cudaEventRecord(b->ev, c->stream));
    DM_BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev, 0));
  }
  for (int it = 0; it < n_iter; ++it) {
    bool graph_ok = b->use_graph;
    std::vector<int> key;
    for (dm_ctx* c : b->ctx) {
      graph_ok = graph_ok && !c->timing && c->iters >= c->p.probe_update_start;
      key.push_back(c->cur_O * 2 + c->cur_P + (use_cluster(c) ? 4 : 0));   // buffers and form
    }
    if (graph_ok) {
      cudaGraphExec_t g = nullptr;
      for (auto& kv : b->graphs)
        if (kv.first == key) g = kv.second;
      if (!g) {
        DM_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_batch_iteration(b);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        DM_BCUDA(b, e);
        const cudaError_t e2 = cudaGraphInstantiate(&g, graph, 0);
        cudaGraphDestroy(graph);
        DM_BCUDA(b, e2);
        b->graphs.emplace_back(key, g);
      }
      DM_BCUDA(b, cudaGraphLaunch(g, b->stream));
    } else {
      const int rc = enqueue_batch_iteration(b);
      if (rc) return rc;
    }
    for (dm_ctx* c : b->ctx) {
      const bool upd = c->iters >= c->p.probe_update_start;
      c->cur_O ^= 1;
      if (upd) c->cur_P ^= 1;
      c->iters++;
    }
  }
  // and every context's stream follows the batch
  DM_BCUDA(b, cudaEventRecord(b->ev, b->stream));
  for (dm_ctx* c : b->ctx) DM_BCUDA(b, cudaStreamWaitEvent(c->stream, b->ev, 0));
  return DM_OK;
}

int dm_batch_set_graph(dm_batch* b, int32_t enable) {
  if (!b) return DM_EINVAL;
  b->use_graph = enable != 0;
  return DM_OK;
}

void dm_batch_free(dm_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (size_t i = 0; i < b->lanes.size(); ++i) {
    if (b->lanes[i]) { cudaStreamSynchronize(b->lanes[i]); cudaStreamDestroy(b->lanes[i]); }
    if (b->joins[i]) cudaEventDestroy(b->joins[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->begin) cudaEventDestroy(b->begin);
  if (b->dispensers) cudaFreeAsync(b->dispensers, b->stream);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* dm_batch_last_error(const dm_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

int dm_set_graph(dm_ctx* c, int32_t enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->use_graph = enable != 0;
  return DM_OK;
}

int dm_run_step(dm_ctx* c, int32_t step) {
  int rc = check_ctx(c);
  if (rc) return rc;
  switch (step) {
    case DM_STEP_FOURIER:
      return run_fourier(c);
    case DM_STEP_OBJECT: {
      {
        Timed t(c, DM_KERNEL_OTHER);
        DM_CUDA(c, dmk::launch_obj_source(c->cview, psi_cur(c), c->half ? 1 : 0, c->probe[c->cur_P], c->N, c->M, c->J,
                                             c->stream));
      }
      if ((rc = run_object(c))) return rc;
      c->cur_O ^= 1;
      return DM_OK;
    }
    case DM_STEP_PROBE:
      if ((rc = run_probe(c, c->obj[c->cur_O]))) return rc;
      c->cur_P ^= 1;
      return DM_OK;
    default:
      return fail(c, DM_EINVAL, "unknown step");
  }
}

int dm_object_partials(dm_ctx* c, float* num, double* den, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!num || !den || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad output");
  const size_t hw = (size_t)c->H * c->W;
  if (!c->den64_O && (rc = alloc_n(c, &c->den64_O, hw))) return rc;
  if ((rc = run_object_gather(c, c->den64_O))) return rc;
  if ((rc = copy_out(c, num, c->num_O, hw * sizeof(float2), mem_kind))) return rc;
  if ((rc = copy_out(c, den, c->den64_O, hw * sizeof(double), mem_kind))) return rc;
  return check_status(c);
}

int dm_object_apply(dm_ctx* c, const double* num, const double* den, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!num || !den || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad input");
  const size_t hw = (size_t)c->H * c->W;
  if (!c->den64_O && (rc = alloc_n(c, &c->den64_O, hw))) return rc;
  if (!c->num64_O && (rc = alloc_n(c, &c->num64_O, hw))) return rc;
  if (!c->dmax64_O && (rc = alloc_n(c, &c->dmax64_O, 1))) return rc;
  if ((rc = copy_in(c, c->num64_O, num, hw * sizeof(double2), mem_kind))) return rc;
  if ((rc = copy_in(c, c->den64_O, den, hw * sizeof(double), mem_kind))) return rc;
  DM_CUDA(c, cudaMemsetAsync(c->dmax64_O, 0, sizeof(unsigned long long), c->stream));
  DM_CUDA(c, dmk::launch_max_f64(c->den64_O, hw, c->dmax64_O, c->stream));
  dmk::ObjFinal64Args f{};
  f.H = c->H; f.W = c->W; f.delta_rel = c->p.denom_floor_rel;
  f.num = c->num64_O; f.den = c->den64_O; f.den_max_bits = c->dmax64_O;
  f.o_start = c->obj[c->cur_O]; f.o_new = c->obj[c->cur_O ^ 1]; f.part = c->obj_part;
  {
    Timed t(c, DM_KERNEL_OBJECT_FINAL);
    DM_CUDA(c, dmk::launch_obj_final64(f, c->obj_final_blocks, c->stream));
  }
  c->cur_O ^= 1;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));   // the inputs may be host temporaries of the caller
  return DM_OK;
}

int dm_probe_partials(dm_ctx* c, double* num, double* den, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!num || !den || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad output");
  // after dm_object_apply the new object is current; Jacobi takes the old one
  if ((rc = run_probe_sums(c, c->obj[c->p.update_order == DM_ORDER_JACOBI ? c->cur_O ^ 1 : c->cur_O]))) return rc;
  const size_t nn = (size_t)c->N * c->N;
  if ((rc = copy_out(c, num, c->num_sum, 2 * (size_t)c->M * nn * sizeof(double), mem_kind))) return rc;
  if ((rc = copy_out(c, den, c->den_sum, nn * sizeof(double), mem_kind))) return rc;
  return check_status(c);
}

int dm_probe_apply(dm_ctx* c, const double* num, const double* den, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!num || !den || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad input");
  const size_t nn = (size_t)c->N * c->N;
  if ((rc = copy_in(c, c->num_sum, num, 2 * (size_t)c->M * nn * sizeof(double), mem_kind))) return rc;
  if ((rc = copy_in(c, c->den_sum, den, nn * sizeof(double), mem_kind))) return rc;
  DM_CUDA(c, cudaMemsetAsync(c->dmax_P, 0, sizeof(unsigned long long), c->stream));
  DM_CUDA(c, dmk::launch_max_f64(c->den_sum, nn, c->dmax_P, c->stream));
  if ((rc = run_probe_div(c))) return rc;
  c->cur_P ^= 1;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}

int dm_fourier_error_partials(dm_ctx* c, double* sums) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!sums) return fail(c, DM_EINVAL, "sums is NULL");
  DM_CUDA(c, dmk::launch_reduce_sum(c->ef_part, (long long)c->J * c->ef_cg, 1, 0, c->ef_tot, c->stream));
  DM_CUDA(c, cudaMemcpyAsync(c->ef_tot + 1, c->isum, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if ((rc = copy_out(c, sums, c->ef_tot, 2 * sizeof(double), DM_HOST))) return rc;
  return check_status(c);
}

int dm_finish_iteration(dm_ctx* c, const double* sums) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!sums) return fail(c, DM_EINVAL, "sums is NULL");
  if ((rc = copy_in(c, c->ef_tot, sums, 2 * sizeof(double), DM_HOST))) return rc;
  if ((rc = run_metrics(c, c->ef_tot, 1, c->ef_tot + 1, true, false))) return rc;
  c->iters++;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}

int dm_get_object(dm_ctx* c, float* out, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad output");
  if ((rc = copy_out(c, out, c->obj[c->cur_O], (size_t)c->H * c->W * sizeof(float2), mem_kind))) return rc;
  return check_status(c);
}

int dm_get_probe(dm_ctx* c, float* out, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad output");
  if ((rc = copy_out(c, out, c->probe[c->cur_P], (size_t)c->M * c->N * c->N * sizeof(float2), mem_kind))) return rc;
  return check_status(c);
}

int dm_get_exit_waves(dm_ctx* c, float* out, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad output");
  const size_t n = (size_t)c->J * c->M * c->N * c->N;
  // the half form is widened into the complex64 buffer first (exactly: every half is a float)
  if (c->half) DM_CUDA(c, dmk::launch_psi_convert(c->psi, c->psi16, n, 0, c->stream));
  if ((rc = copy_out(c, out, c->psi, n * sizeof(float2), mem_kind))) return rc;
  return check_status(c);
}

int dm_set_exit_waves(dm_ctx* c, const float* in, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!in || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad input");
  const size_t n = (size_t)c->J * c->M * c->N * c->N;
  if ((rc = copy_in(c, c->psi, in, n * sizeof(float2), mem_kind))) return rc;
  // the half form keeps the values rounded to complex half
  if (c->half) DM_CUDA(c, dmk::launch_psi_convert(c->psi16, c->psi, n, 1, c->stream));
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}


int dm_set_object(dm_ctx* c, const float* in, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!in || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad input");
  if ((rc = copy_in(c, c->obj[c->cur_O], in, (size_t)c->H * c->W * sizeof(float2), mem_kind))) return rc;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}

int dm_set_probe(dm_ctx* c, const float* in, int32_t mem_kind) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!in || (mem_kind != DM_HOST && mem_kind != DM_DEVICE)) return fail(c, DM_EINVAL, "bad input");
  if ((rc = copy_in(c, c->probe[c->cur_P], in, (size_t)c->M * c->N * c->N * sizeof(float2), mem_kind))) return rc;
  DM_CUDA(c, dmk::launch_p2(c->p2, c->probe[c->cur_P], c->N, c->M, c->stream));
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DM_OK;
}

int dm_get_error(dm_ctx* c, int32_t iter, double* eps_obj, double* eps_probe, double* fourier_err) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (c->iters == 0) return fail(c, DM_EINVAL, "no iteration has run");
  const int64_t it = iter < 0 ? c->iters - 1 : iter;
  if (it >= c->iters || it < c->iters - dmk::kMetricsRing || it < 0)
    return fail(c, DM_EINVAL, "iteration not available");
  double row[2 + dmk::kMaxModes];
  const size_t bytes = sizeof(double) * (2 + c->M);
  DM_CUDA(c, cudaMemcpyAsync(row, c->ring + (size_t)(it % dmk::kMetricsRing) * dmk::kRingRow, bytes,
                             cudaMemcpyDeviceToHost, c->stream));
  if ((rc = check_status(c))) return rc;
  if (eps_obj) *eps_obj = row[0];
  if (fourier_err) *fourier_err = row[1];
  if (eps_probe) for (int k = 0; k < c->M; ++k) eps_probe[k] = row[2 + k];
  return DM_OK;
}

int dm_set_psi_error(dm_ctx* c, int32_t enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (enable && c->half) return fail(c, DM_EINVAL, "the exit-wave change is tracked with complex64 exit waves only");
  DM_CUDA(c, cudaStreamSynchronize(c->stream));   // no captured iteration is in flight below
  if (enable && !c->psi_part && (rc = alloc_n(c, &c->psi_part, (size_t)c->J * c->fa.RB * 2))) return rc;
  c->psi_err = enable != 0;
  c->fa.psi_part = c->psi_err ? c->psi_part : nullptr;
  // captured iterations hold the previous Fourier-step instance
  for (auto& row : c->gexec)
    for (auto& g : row)
      if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  return DM_OK;
}

int dm_get_psi_error(dm_ctx* c, int32_t iter, double* eps_psi) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!eps_psi) return fail(c, DM_EINVAL, "eps_psi is NULL");
  if (c->iters == 0) return fail(c, DM_EINVAL, "no iteration has run");
  const int64_t it = iter < 0 ? c->iters - 1 : iter;
  if (it >= c->iters || it < c->iters - dmk::kMetricsRing || it < 0)
    return fail(c, DM_EINVAL, "iteration not available");
  DM_CUDA(c, cudaMemcpyAsync(eps_psi, c->ring + (size_t)(it % dmk::kMetricsRing) * dmk::kRingRow + dmk::kRingPsi,
                             sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_status(c);
}

int dm_selftest_bounded_waits(double* elapsed_ms) {
  g_init_error.clear();
  int* d = nullptr;   // [0] flag nothing raises, [1..2] status words, [3..4] wait results
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d), 5 * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc");
  int h[5] = {0, 0, 0, 0, 0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  e = cudaMemset(d, 0, 5 * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  if (e == cudaSuccess) e = dmk::launch_wait_selftest(d, d + 1, d + 3, 0);
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  // the context is still usable: a plain device operation after the waits
  if (e == cudaSuccess) e = cudaMemset(d, 0, 5 * sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "bounded-wait self-test");
  if (elapsed_ms) *elapsed_ms = ms;
  const bool gave_up = h[3] == 0 && h[4] == 0;
  const bool flagged = (h[1] & dmk::kStatusTimeout) && (h[2] & dmk::kStatusTimeout);
  if (!gave_up || !flagged) return fail(nullptr, DM_EINVAL, "a bounded wait did not give up as designed");
  return DM_OK;
}

int64_t dm_iterations_done(const dm_ctx* c) { return c ? c->iters : -1; }

int dm_get_mode_power(dm_ctx* c, double* out) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!out) return fail(c, DM_EINVAL, "out is NULL");
  DM_CUDA(c, dmk::launch_mode_power(c->probe[c->cur_P], c->N, c->M, c->mode_pow, c->stream));
  DM_CUDA(c, cudaMemcpyAsync(out, c->mode_pow, sizeof(double) * c->M, cudaMemcpyDeviceToHost, c->stream));
  return check_status(c);
}

int dm_sync(dm_ctx* c) {
  int rc = check_ctx(c);
  if (rc) return rc;
  DM_CUDA(c, cudaStreamSynchronize(c->stream));
  DM_CUDA(c, cudaGetLastError());
  return check_status(c);
}

int dm_set_timing(dm_ctx* c, int32_t enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = collect_timing(c))) return rc;
  for (int k = 0; k < DM_KERNEL_COUNT; ++k) { c->kms[k] = 0.0; c->klaunch[k] = 0; }
  c->timing = enable != 0;
  return DM_OK;
}

int dm_get_timing(dm_ctx* c, int32_t kernel, double* total_ms, int64_t* launches) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (kernel < 0 || kernel >= DM_KERNEL_COUNT) return fail(c, DM_EINVAL, "unknown kernel class");
  if ((rc = collect_timing(c))) return rc;
  if (total_ms) *total_ms = c->kms[kernel];
  if (launches) *launches = c->klaunch[kernel];
  return DM_OK;
}

const char* dm_kernel_name(int32_t kernel) {
  static const char* names[DM_KERNEL_COUNT] = {"fourier",       "object_gather", "object_final", "probe_partial",
                                               "probe_final",   "metrics",       "other"};
  return (kernel >= 0 && kernel < DM_KERNEL_COUNT) ? names[kernel] : "unknown";
}

size_t dm_device_bytes(const dm_ctx* c) { return c ? c->bytes : 0; }

void dm_free(dm_ctx* c) {
  if (!c || c->magic != 0x58434D44u) return;
  c->magic = 0;
  cudaSetDevice(c->device);
  release_all(c);
  delete c;
}

const char* dm_last_error(const dm_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

}  // extern "C"
