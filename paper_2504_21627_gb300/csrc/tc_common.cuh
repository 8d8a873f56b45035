// Helpers shared by the fused query kernels (BF16 and FP8): tcgen05
// descriptors and fences, bounded mbarrier waits, TMEM loads, the
// no-swizzle K-major core-matrix layout and the per-tile work-list rule.
#pragma once

#include <cstdint>

#include "lsnif_impl.h"

namespace lsnif {
namespace {

constexpr int kListStride = 2 * kTileM;  // work-list entries per chunk: two per ray
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t addr, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// One test of the phase; a thread whose phase is not complete is suspended
// (it issues nothing) until the phase completes or about 0.1 ms pass.
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(parity), "r"(100000)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of the given parity. Gives up at once when
// another thread has flagged an abort, and flags one itself on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, volatile int *abort_flag) {
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(addr, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
}

// The same with a sleep between tests (32 ns doubling to 512 ns), for
// kernels whose waiting warps share the SM's issue slots with busy ones: a
// waiting warp then issues fewer instructions. In the fused query kernel
// this was 1% faster than waking on every completed test.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t addr, uint32_t parity, volatile int *abort_flag) {
  const long long t0 = clock64();
  unsigned ns = 32u;
  while (true) {
    if (mbar_try(addr, parity)) return true;
    __nanosleep(ns);
    ns = ns < 512u ? 2u * ns : 512u;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag (teardown: in-flight MMAs).
__device__ __forceinline__ bool mbar_wait_teardown(uint32_t addr, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(addr, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}


// named barrier among `count` threads (id 0 is __syncthreads)
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

#define TMEM_LD16(taddr, r)                                                                                        \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
               "[%16];"                                                                                            \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),         \
                 "=r"(r[15])                                                                                       \
               : "r"(taddr))

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 consecutive 32-bit TMEM columns of the warp's 32 lanes from registers
// (thread i writes lane i of the warp's lane quarter)
#define TMEM_ST8(taddr, r)                                                                                   \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),    \
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])  \
               : "memory")

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// byte offset of the 16-byte row piece (row r, core K-group kg of 16 bytes)
// in a tile of 8-row core matrices with row-group stride sbo
__device__ __forceinline__ uint32_t core_off(int r, int kg, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(r & 7) * 16u;
}

struct TileInfo {
  int32_t kmax, slot, stop, pad;
};

__host__ __device__ inline uint32_t lay_take(uint32_t &off, uint32_t bytes, uint32_t align) {
  off = (off + align - 1) & ~(align - 1);
  const uint32_t r = off;
  off += bytes;
  return r;
}

// work-list counts of one ray for chunk s, packed: gathers | copies << 10 |
// zero fills << 20 (always two entries per ray)
__device__ __forceinline__ uint32_t row_counts(int kk, uint32_t dm, int s) {
  if (kk <= s) return 2u << 20;
  const bool dup = s > 0 && ((dm >> s) & 1u);
  return dup ? (1u | (1u << 10)) : 2u;
}

}  // namespace
}  // namespace lsnif
