// Encoders of the two descriptors a tcgen05.mma takes (PTX ISA, "tcgen05"
// chapter: the instruction descriptor and the shared-memory matrix
// descriptor).  Plain C++ so that a host test can check the bit fields
// without a GPU; the device code includes the same header.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define DM_TC05_HD __host__ __device__
#else
#define DM_TC05_HD
#endif

namespace dmtc {

// Operand and accumulator formats of kind::f16 (D: F16 0, F32 1; A and B:
// F16 0, BF16 1).
enum : uint32_t { kFmtF16 = 0, kFmtF32 = 1, kFmtBF16 = 1 };

// Instruction descriptor of tcgen05.mma.kind::f16, dense, no negation:
//   bits  4-5  D format          bits  7-9  A format     bits 10-12 B format
//   bit  15    A transposed (0: K-major)   bit 16 B transposed (0: K-major)
//   bits 17-22 N / 8             bits 24-28 M / 16
// (bits 0-3 sparsity and saturation, 13-14 negation, 23 and 29 reserved,
// 30-31 the weight-stationary shift: all 0 here).
DM_TC05_HD constexpr uint32_t idesc_f16(uint32_t d_fmt, uint32_t a_fmt, uint32_t b_fmt, uint32_t m, uint32_t n,
                                        bool a_mn_major = false, bool b_mn_major = false) {
  return (d_fmt << 4) | (a_fmt << 7) | (b_fmt << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((b_mn_major ? 1u : 0u) << 16) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Swizzle modes of the shared-memory descriptor (bits 61-63).
enum : uint64_t { kSwNone = 0, kSw128B32 = 1, kSw128 = 2, kSw64 = 4, kSw32 = 6 };

// Shared-memory matrix descriptor:
//   bits  0-13 start address / 16 (shared-window address, 18 bits used)
//   bits 16-29 leading-dimension byte offset / 16
//   bits 32-45 stride-dimension byte offset / 16
//   bits 46-48 the fixed value 0b001
//   bits 49-51 base offset (0: the swizzle pattern starts at a boundary of
//              its repeat)    bit 52 leading-offset mode (0: relative)
//   bits 61-63 swizzle mode
DM_TC05_HD constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes, uint64_t swizzle) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (swizzle << 61);
}

// TMEM address of (lane, column): lane in bits 16-31, column in bits 0-15.
DM_TC05_HD constexpr uint32_t tmem_addr(uint32_t base, uint32_t lane, uint32_t col) {
  return base + (lane << 16) + col;
}

}  // namespace dmtc
