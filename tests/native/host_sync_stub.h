// host_sync_stub.h -- host stand-ins for fp_sync.cuh's PTX helpers, for the
// block emulation of the parse kernel (tests/native/parse_block_emu.cpp): the
// emulated threads run one at a time, so plain loads and stores are
// ordered; a bulk copy completes when it is issued (so every mbarrier
// phase has completed by the time anyone waits on it); the timer is the
// host's monotonic clock.  The test copies this file next to the kernel
// header as fp_sync.cuh.
#pragma once
#include <chrono>
#include <cstdint>
#include <cstring>

namespace fp {

inline void st_relaxed_u64(unsigned long long* p, unsigned long long v) { *p = v; }
inline unsigned long long ld_relaxed_u64(const unsigned long long* p) { return *p; }
inline void st_release_u64(unsigned long long* p, unsigned long long v) { *p = v; }
inline unsigned long long ld_acquire_u64(const unsigned long long* p) { return *p; }
inline uint64_t globaltimer_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}
inline void mbar_init(uint64_t* bar, uint32_t) { *bar = 0; }
inline void fence_mbar_init() {}
inline void mbar_arrive_expect_tx(uint64_t*, uint32_t) {}
inline void mbar_arrive(uint64_t*) {}
inline bool mbar_try_wait(uint64_t*, uint32_t) { return true; }
inline void fence_proxy_async_smem() {}
inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t*) {
  std::memcpy(dst, src, bytes);
}
inline void grid_launch_dependents() {}
inline void grid_dependency_wait() {}

}  // namespace fp
