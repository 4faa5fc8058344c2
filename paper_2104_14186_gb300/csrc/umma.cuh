// Shared building blocks of the library's tcgen05 (5th-generation tensor core) kernels: TMA
// tiled loads, shared-memory matrix descriptors, tensor-memory loads, bounded mbarrier waits,
// and the tensor maps of bfloat16 "slice" arrays.  Used by the emulated-FP64 digit products
// (ozaki.cu) and the FP32-accurate split products (bf16x6.cu).
//
// Slice arrays are [slice][rows_pad][k_pad] bfloat16 with K contiguous, zero padded to
// 128-row blocks; a TMA box is 64 (K) x 128 (rows) x 1 slice, i.e. one 128-byte swizzle atom
// column of 16 KB, written by the copy engine in the layout the MMA descriptors below expect
// (K-major, 8-row atoms of 1024 bytes, 16-byte chunk c of row r at chunk c ^ (r % 8)).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "internal.h"

namespace qdwhp {
namespace umma {

constexpr int kAtomK = 64;                                 // K of one 128-byte swizzle atom row (bf16)
constexpr uint32_t kAtomBytes = 128 * kAtomK * 2;          // 16 KB: 128 rows x 64 K
constexpr int kSpin = 1 << 24;                             // bound of every mbarrier wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, leading byte offset 16 (unused with swizzle),
// stride byte offset 1024 (next 8-row atom), descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of tcgen05.mma kind::f16 with BF16 A and B, FP32 accumulation, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// D (TMEM) += or = A (smem descriptor) x B (smem descriptor), one tcgen05.mma of shape idesc.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
               : "r"(taddr));
}

// Waits for the phase `parity` of the mbarrier, at most kSpin polls; gives up early once
// *abort_flag is set (another thread of the CTA gave up).  false = the wait gave up.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (int it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}

// The same for waiters off the critical path: sleeps ~100 ns after each failed poll, so that
// the warp takes no issue slots from the threads that feed the tensor cores; at most kSpinSleep
// polls (about half a second or more).
constexpr int kSpinSleep = 1 << 22;
__device__ __forceinline__ bool mbar_wait_sleep_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (int it = 0; it < kSpinSleep; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63 && *abort_flag) return false;
    __nanosleep(100);
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Tensor map of a [nslices][rows_pad][k_pad] bfloat16 slice array (k innermost; k_pad a multiple
// of 64, rows_pad of 128), box 64 x 128 x 1 with the 128-byte swizzle.
qdwhp_status slice_map(CUtensorMap* map, const unsigned short* base, int nslices, int rows_pad, int k_pad);

}  // namespace umma
}  // namespace qdwhp
