// The 256-point row DFT as one dense complex GEMM on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory), the third
// precision form of dm_dft2 (DM_DFT_BF16X3_TC05).
//
// A row x of 256 complex values is, as stored, 512 floats (re, im
// interleaved).  With the same interleaving of the output,
//   X[q] = sum_k x[k] W^(kq),  W = exp(-+2 pi i / 256),  W^(kq) = c + i s,
// is the real product D = A B of the row (K = 512) with the 512 x 512 real
// matrix B[2k][2q] = c, B[2k+1][2q] = -s, B[2k][2q+1] = s, B[2k+1][2q+1] = c.
// A CTA takes 128 rows (M = 128) and the full N = 512 in two halves of 256
// tensor-memory columns each.  Both operands are split a = hi + lo into BF16
// (hi = bf16(a), lo = bf16(a - hi)) and each product is hi*hi + hi*lo +
// lo*hi, with FP32 accumulation; the dropped lo*lo term is 2^-16 of a
// product.  Compared with the two radix-16 stages of the mma.sync form this
// does 16 times the arithmetic, but it has no twiddle step and no transpose
// between stages, and the tensor cores have the arithmetic to spare.
//
// Data movement: the B planes (hi and lo, both directions) are a device
// table streamed by TMA in the 64-byte-swizzled K-major layout, 32 K values
// per pipeline stage in a ring of four; four producer warps (one thread per row) load the
// rows' FP32 values, split them and write A in the same layout; one thread
// issues the MMAs and the TMA loads; the producer warps then read the
// accumulators back (tcgen05.ld, lane = row) and store them transposed, one
// coalesced row of the output per column pair.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dm_kernels.h"
#include "dm_ptx.cuh"
#include "dm_tc05_desc.h"

namespace dmk {

namespace {

constexpr int kTN = 256;                  // transform length
constexpr int kTK = 2 * kTN;              // real K (= real N) of the GEMM
constexpr int kTM = 128;                  // rows per CTA (MMA M)
constexpr int kTNh = 256;                 // MMA N (half of the output columns)
constexpr int kStageK = 32;               // real K per pipeline stage (one 64-byte swizzle row)
constexpr int kStages = kTK / kStageK;    // 16 stages per N half
constexpr int kRing = 4;                  // stage buffers
constexpr int kRowB = kStageK * 2;        // bytes of one operand row in a stage (the swizzle span)
constexpr int kAtomB = 8 * kRowB;         // bytes of one 8-row swizzle atom (the MMA's stride offset)
constexpr int kABytes = kTM * kStageK * 2;     // 8 KB: one A plane of a stage
constexpr int kBBytes = kTNh * kStageK * 2;    // 16 KB: one B plane of a stage
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;   // A hi, A lo, B hi, B lo
constexpr int kProducers = 128;           // producer threads (warps 0-3)
constexpr int kEpilogue = 128;            // epilogue threads (warps 5-8)
constexpr int kTcThreads = kProducers + 32 + kEpilogue;   // + the MMA warp (warp 4)
constexpr size_t kTcSmem = 1024 + (size_t)kRing * kStageBytes;

// B planes: [direction][hi, lo][n][k] as BF16, n the real output index and
// k the real input index (K-major rows of 512 values).
__device__ __nv_bfloat16 g_tc_b[2][2][kTK][kTK];
__device__ int g_tc_status;   // kStatusTimeout once a bounded wait of the kernel gave up

__global__ void k_tc_tables() {
  const int n = blockIdx.x, dir = blockIdx.y;   // grid (512, 2), 256 threads
  const int q = n >> 1, po = n & 1;
  for (int kk = threadIdx.x; kk < kTK; kk += blockDim.x) {
    const int k = kk >> 1, pi = kk & 1;
    double s, c;
    sincospi(2.0 * (double)((k * q) % kTN) / kTN, &s, &c);   // angle 2 pi k q / 256
    const double sg = dir ? s : -s;                            // W^(kq) = c + i sg
    // rows of B: input (k, pi), columns: output (q, po)
    const double v = po == 0 ? (pi == 0 ? c : -sg) : (pi == 0 ? sg : c);
    const __nv_bfloat16 h = __double2bfloat16(v);
    g_tc_b[dir][0][n][kk] = h;
    g_tc_b[dir][1][n][kk] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

// ---- tcgen05 and TMEM (PTX ISA, tcgen05 chapter) --------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tmem) = A B (+ D when acc), one thread.
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
      : "memory");
}

// The mbarrier gets one arrival when every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive 32-bit columns of this thread's lane (the warp's quarter of
// the 128 lanes), then the wait for the load.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait that records a timeout in g_tc_status.
__device__ __forceinline__ void tc_wait(uint64_t* bar, uint32_t parity) {
  (void)mbar_wait_bounded(bar, parity, &g_tc_status);
}

// Eight floats (one 16-byte chunk of K values) split into BF16 hi and lo.
__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // a in the low half
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void split8(const float4& u, const float4& w, uint4& hi, uint4& lo) {
  const float x[8] = {u.x, u.y, u.z, u.w, w.x, w.y, w.z, w.w};
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = bf2(x[2 * i], x[2 * i + 1]);
    const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&h[i]);
    const float2 hf = __bfloat1622float2(hv);
    l[i] = bf2(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// One pass: the 256-point DFT of every 128-row tile (rows r0.. of frame f),
// stored transposed (out[f][q][r]).  Persistent: CTA c takes tiles c, c +
// grid, ...  Warps 0-3 produce A; warp 4 allocates tensor memory and its
// lane 0 issues the B loads and the MMAs; warps 5-8 read the accumulators
// back (warp w reads tensor-memory lanes 32 (w % 4) .., thread = row) and
// store them.  Each N half has its own 256 accumulator columns with a full
// and an empty barrier, so one half is drained while the MMAs of the other
// half (or of the next tile) run.
template <bool INV>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_dft256_rows_tc05(const __grid_constant__ CUtensorMap tmB, const float2* __restrict__ in,
                       float2* __restrict__ out, int ntiles) {
  extern __shared__ unsigned char tc_raw[];
  // 1024-byte aligned stages (the 64-byte swizzle repeats every 512 bytes)
  unsigned char* base = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full[kRing], empty[kRing], accf[2], acce[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == kProducers) {
    for (int b = 0; b < kRing; ++b) {
      mbar_init(&full[b], kProducers + 1);   // the producers and the B loads' expect_tx
      mbar_init(&empty[b], 1);               // the MMA thread's commit
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&accf[h], 1);                // the MMA thread's commit: half h complete
      mbar_init(&acce[h], kEpilogue);        // the epilogue threads: half h drained
    }
    fence_mbar_init();
  }
  if (warp == 4) tmem_alloc(&s_tmem, 2 * kTNh);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr uint32_t idesc = dmtc::idesc_f16(dmtc::kFmtF32, dmtc::kFmtBF16, dmtc::kFmtBF16, kTM, kTNh);
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nst = my_tiles * 2 * kStages;   // pipeline stages of this CTA

  if (warp < 4) {
    // ---- producers: the A planes of every stage ----
    // Chunk task i (of 512 per stage: 128 rows x 4 chunks of 8 K values) is
    // row i / 4, chunk i % 4; thread t takes tasks t + 128 it, so 4
    // consecutive threads read one row's 128 contiguous bytes (coalesced) and
    // write its 4 chunks (the swizzle spreads them over the banks).
    constexpr int kCh = kStageK / 8;   // chunks per row and stage
    constexpr int kIt = kTM * kCh / kProducers;
    float4 buf[3][2 * kIt];
    auto load = [&](int g, float4 (&d)[2 * kIt]) {
      const int tile = blockIdx.x + (g / (2 * kStages)) * gridDim.x, s = g % kStages;
      const float4* rows = reinterpret_cast<const float4*>(in + (size_t)tile * kTM * kTN);
#pragma unroll
      for (int it = 0; it < kIt; ++it) {
        const int id = it * kProducers + tid, row = id / kCh, j = id % kCh;
        const float4* p = rows + (size_t)row * (kTN / 2) + s * (kStageK / 4) + 2 * j;
        d[2 * it] = __ldg(p);
        d[2 * it + 1] = __ldg(p + 1);
      }
    };
    auto store = [&](int g, const float4 (&d)[2 * kIt]) {
      const int b = g % kRing;
      if (g >= kRing) tc_wait(&empty[b], ((g / kRing) - 1) & 1);   // the MMAs of stage g - kRing are done
      unsigned char* ah = base + (size_t)b * kStageBytes;
#pragma unroll
      for (int it = 0; it < kIt; ++it) {
        const int id = it * kProducers + tid, row = id / kCh, j = id % kCh;
        uint4 hi, lo;
        split8(d[2 * it], d[2 * it + 1], hi, lo);
        // 64-byte swizzle: 16-byte chunk ^ bits 7-8 of the row's offset
        const int off = row * kRowB + ((j ^ ((row >> 1) & 3)) << 4);
        *reinterpret_cast<uint4*>(ah + off) = hi;
        *reinterpret_cast<uint4*>(ah + kABytes + off) = lo;
      }
      fence_proxy_async_smem();   // visible to the tensor cores (async proxy)
      mbar_arrive(&full[b]);
    };
    // loads run two stages ahead of the stores (three register buffers,
    // rotated by unrolling three stages per trip; written out by hand: a
    // generic unrolled loop of the same order measured 10 % slower, and
    // three or four stages ahead slower still)
    if (nst > 0) load(0, buf[0]);
    if (nst > 1) load(1, buf[1]);
    for (int g = 0; g < nst; g += 3) {
      if (g + 2 < nst) load(g + 2, buf[2]);
      store(g, buf[0]);
      if (g + 1 < nst) {
        if (g + 3 < nst) load(g + 3, buf[0]);
        store(g + 1, buf[1]);
      }
      if (g + 2 < nst) {
        if (g + 4 < nst) load(g + 4, buf[1]);
        store(g + 2, buf[2]);
      }
    }
  } else if (warp == 4) {
    if (lane == 0) {
      // ---- B loads and MMAs (one thread) ----
      const uint64_t pol = l2_policy_evict_last();
      const int plane = INV ? 2 : 0;
      auto load_b = [&](int g) {
        const int b = g % kRing, s = g % kStages, h = (g / kStages) & 1;
        unsigned char* bh = base + (size_t)b * kStageBytes + 2 * kABytes;
        mbar_arrive_expect_tx(&full[b], 2 * kBBytes);
        tma_load_3d_hint(bh, &tmB, s * kStageK, h * kTNh, plane, &full[b], pol);
        tma_load_3d_hint(bh + kBBytes, &tmB, s * kStageK, h * kTNh, plane + 1, &full[b], pol);
      };
      if (nst > 0) load_b(0);
      for (int g = 0; g < nst; ++g) {
        const int b = g % kRing, s = g % kStages, h = (g / kStages) & 1, i = g / (2 * kStages);
        if (g + 1 < nst) {
          // the next stage's buffer held stage g + 1 - kRing: its MMAs must be done
          if (g + 1 >= kRing) tc_wait(&empty[(g + 1) % kRing], (((g + 1) / kRing) - 1) & 1);
          load_b(g + 1);
        }
        if (s == 0 && i > 0) {   // half h of the previous tile has been drained
          tc_wait(&acce[h], (i - 1) & 1);
          tc_fence_after();
        }
        tc_wait(&full[b], (g / kRing) & 1);
        tc_fence_after();
        const uint32_t sa = smem_u32(base + (size_t)b * kStageBytes);
        const uint32_t d = tmem + (uint32_t)(h * kTNh);
#pragma unroll
        for (int kk = 0; kk < kStageK / 16; ++kk) {
          const uint32_t o = 32u * kk;   // 16 BF16 K values further along the swizzle row
          const uint64_t ahd = dmtc::smem_desc(sa + o, 16, kAtomB, dmtc::kSw64);
          const uint64_t ald = dmtc::smem_desc(sa + kABytes + o, 16, kAtomB, dmtc::kSw64);
          const uint64_t bhd = dmtc::smem_desc(sa + 2 * kABytes + o, 16, kAtomB, dmtc::kSw64);
          const uint64_t bld = dmtc::smem_desc(sa + 2 * kABytes + kBBytes + o, 16, kAtomB, dmtc::kSw64);
          tc_mma_f16(d, ahd, bhd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
          tc_mma_f16(d, ahd, bld, idesc, 1u);
          tc_mma_f16(d, ald, bhd, idesc, 1u);
        }
        tc_commit(&empty[b]);
        if (s == kStages - 1) tc_commit(&accf[h]);   // half h of this tile is complete
      }
      // every MMA has completed before the tensor memory is freed (already so
      // unless a bounded wait above gave up)
      if (nst > 0) tc_wait(&empty[(nst - 1) % kRing], ((nst - 1) / kRing) & 1);
    }
  } else {
    // ---- epilogue: accumulators back, stored transposed ----
    const int q4 = warp & 3, r = 32 * q4 + lane;   // tensor-memory lane = row of the tile
    for (int i = 0; i < my_tiles; ++i) {
      const int tile = blockIdx.x + i * gridDim.x;
      const int f = tile >> 1, r0 = (tile & 1) * kTM;
      float2* dst = out + (size_t)f * kTN * kTN + r0 + r;
      for (int h = 0; h < 2; ++h) {
        tc_wait(&accf[h], i & 1);
        tc_fence_after();
        for (int cc = 0; cc < kTNh / 32; ++cc) {
          float v[32];
          tmem_ld32(dmtc::tmem_addr(tmem, 32 * q4, h * kTNh + 32 * cc), v);
          const int q0 = (h * kTNh + 32 * cc) / 2;
#pragma unroll
          for (int e = 0; e < 16; ++e) __stcs(dst + (size_t)(q0 + e) * kTN, make_float2(v[2 * e], v[2 * e + 1]));
        }
        tc_fence_before();
        mbar_arrive(&acce[h]);
      }
    }
  }
  __syncthreads();
  if (warp == 4) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * kTNh);
  }
}

}  // namespace

// The B table, its TMA view and the kernels' shared-memory limit, once per
// device (the caller holds a lock).
static CUtensorMap g_tc_map[64];

cudaError_t prepare_dft256_tc05(cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  for (const void* f : {(const void*)k_dft256_rows_tc05<false>, (const void*)k_dft256_rows_tc05<true>}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
  }
  k_tc_tables<<<dim3(kTK, 2), 256, 0, s>>>();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  void* table = nullptr;
  if ((e = cudaGetSymbolAddress(&table, g_tc_b)) != cudaSuccess) return e;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (!fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  // [plane][n][k] BF16: dims (k, n, plane), box 64 k x 256 n x 1 plane
  const cuuint64_t dims[3] = {(cuuint64_t)kTK, (cuuint64_t)kTK, 4};
  const cuuint64_t strides[2] = {(cuuint64_t)kTK * 2, (cuuint64_t)kTK * kTK * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kStageK, (cuuint32_t)kTNh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(&g_tc_map[dev], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, table, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_dft256_tc05(const float2* in, float2* work, float2* out, int frames, bool inverse,
                               cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const CUtensorMap& m = g_tc_map[dev];
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int ntiles = 2 * frames;                    // 128-row tiles per pass
  const int grid = ntiles < sms ? ntiles : sms;     // persistent, one CTA per SM
  for (int pass = 0; pass < 2; ++pass) {
    const float2* a = pass == 0 ? in : work;
    float2* b = pass == 0 ? work : out;
    if (inverse) k_dft256_rows_tc05<true><<<grid, kTcThreads, kTcSmem, s>>>(m, a, b, ntiles);
    else k_dft256_rows_tc05<false><<<grid, kTcThreads, kTcSmem, s>>>(m, a, b, ntiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The status word of the tcgen05 form's bounded waits: read and cleared
// after the device has finished its work.
cudaError_t dft256_tc05_status(int* timed_out) {
  cudaError_t e = cudaDeviceSynchronize();
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int));
  const int zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int));
  *timed_out = (v & kStatusTimeout) ? 1 : 0;
  return e;
}

}  // namespace dmk
