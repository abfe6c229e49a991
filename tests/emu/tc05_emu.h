// Host emulation of the tcgen05 primitives of tc05.cuh (test
// infrastructure), installed under that name when device code is compiled for
// the host. An MMA is carried out when it is issued, reading its operands
// through the decoded shared-memory descriptors (every address checked
// against the block's shared memory) and accumulating in FP32 into an
// emulated tensor memory of 128 lanes x 512 columns; a commit completes the
// mbarrier's phase. Loads check that a warp reads only its own lane quarter.
#pragma once
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_bf16.h>
#include <map>
#include <mutex>
#include <thread>

namespace vio {
namespace tc {

struct EmuTc {
  uint8_t* smem = nullptr;   // the block's shared memory
  size_t smem_bytes = 0;
  float tmem[128][512];
  long mmas = 0;
};
inline EmuTc*& emu_tc() {
  static EmuTc* p = nullptr;
  return p;
}

[[noreturn]] inline void emu_fail(const char* what) {
  fprintf(stderr, "TC EMU: %s\n", what);
  std::abort();
}

inline uint32_t smem_u32(const void* p) {
  const uint8_t* b = static_cast<const uint8_t*>(p);
  if (b < emu_tc()->smem || b >= emu_tc()->smem + emu_tc()->smem_bytes)
    emu_fail("pointer outside shared memory");
  return (uint32_t)(b - emu_tc()->smem);
}

inline uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  if ((addr | lbo | sbo) & 15) emu_fail("descriptor offset not a multiple of 16");
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

inline void tmem_alloc(uint32_t* slot, uint32_t cols) {
  if (cols < 32 || cols > 512 || (cols & (cols - 1))) emu_fail("bad column count");
  if ((threadIdx.x & 31) == 0) *slot = 0;
  __syncwarp();
}
inline void tmem_free(uint32_t, uint32_t) { __syncwarp(); }

inline float emu_bf(const uint8_t* p) {
  uint16_t h;
  memcpy(&h, p, 2);
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

inline void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, bool accumulate) {
  EmuTc& T = *emu_tc();
  const int M = (int)((id >> 24) & 31) * 16, N = (int)((id >> 17) & 63) * 8;
  if (id != idesc_bf16(M, N) || M != 128 || N < 16 || N > 256 || (N & 15))
    emu_fail("unsupported instruction descriptor");
  auto dec = [](uint64_t s, uint32_t& start, uint32_t& lbo, uint32_t& sbo) {
    if (((s >> 46) & 7) != 1 || (s >> 49) != 0) emu_fail("descriptor version or swizzle");
    start = (uint32_t)(s & 0x3fff) << 4;
    lbo = (uint32_t)((s >> 16) & 0x3fff) << 4;
    sbo = (uint32_t)((s >> 32) & 0x3fff) << 4;
  };
  uint32_t as, al, ab, bs, bl, bb;
  dec(a, as, al, ab);
  dec(b, bs, bl, bb);
  auto at = [&](uint32_t start, uint32_t lbo, uint32_t sbo, int row, int k) -> float {
    const size_t off = start + (size_t)(k >> 3) * lbo + (size_t)(row >> 3) * sbo +
                       (row & 7) * 16 + (k & 7) * 2;
    if (off + 2 > T.smem_bytes) emu_fail("operand read outside shared memory");
    return emu_bf(T.smem + off);
  };
  const int lane0 = (int)(d >> 16), col0 = (int)(d & 0xffff);
  if (lane0 != 0 || col0 + N > 512) emu_fail("accumulator outside tensor memory");
  for (int i = 0; i < M; ++i)
    for (int n = 0; n < N; ++n) {
      float s = accumulate ? T.tmem[i][col0 + n] : 0.f;
      for (int k = 0; k < 16; ++k) s += at(as, al, ab, i, k) * at(bs, bl, bb, n, k);
      T.tmem[i][col0 + n] = s;
    }
  ++T.mmas;
}

// The barrier word: completed phases (low 32 bits) and arrivals in the
// current phase (high 32 bits); the expected count is kept beside it.
inline std::atomic<uint64_t>* emu_bar(uint64_t* bar) {
  static_assert(sizeof(std::atomic<uint64_t>) == 8, "barrier word");
  return reinterpret_cast<std::atomic<uint64_t>*>(bar);
}
inline std::mutex& emu_bar_mu() {
  static std::mutex m;
  return m;
}
inline std::map<const void*, uint32_t>& emu_bar_count() {
  static std::map<const void*, uint32_t> m;
  return m;
}
inline void mbar_init(uint64_t* bar, uint32_t count) {
  std::lock_guard<std::mutex> l(emu_bar_mu());
  emu_bar_count()[bar] = count;
  emu_bar(bar)->store(0);
}
inline void fence_mbar_init() {}
inline void mbar_arrive(uint64_t* bar) {
  std::lock_guard<std::mutex> l(emu_bar_mu());
  const uint64_t v = emu_bar(bar)->load();
  const uint32_t arrived = (uint32_t)(v >> 32) + 1, done = (uint32_t)v;
  if (arrived == emu_bar_count()[bar])
    emu_bar(bar)->store((uint64_t)(done + 1));
  else
    emu_bar(bar)->store(((uint64_t)arrived << 32) | done);
}
inline void commit(uint64_t* bar) { mbar_arrive(bar); }   // barriers of count 1
inline void fence_before() {}
inline void fence_after() {}
inline void fence_smem_to_async() {}

// Phase `parity` has completed when the count of completed phases has the
// other parity (waits are for the latest phase). Blocks up to 20 s.
// (not ready: a short sleep, so that a poll limit covers emulated MMA time)
inline bool mbar_try(uint64_t* bar, uint32_t parity) {
  if ((emu_bar(bar)->load() & 1) != parity) return true;
  std::this_thread::sleep_for(std::chrono::microseconds(20));
  return (emu_bar(bar)->load() & 1) != parity;
}
inline bool mbar_wait(uint64_t* bar, uint32_t parity, int) {
  const auto t0 = std::chrono::steady_clock::now();
  while ((emu_bar(bar)->load() & 1) == parity) {
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(20)) return false;
    std::this_thread::yield();
  }
  return true;
}

inline uint32_t taddr(uint32_t base, int lane, int col) {
  return base + ((uint32_t)lane << 16) + (uint32_t)col;
}

template <int NC>
inline void emu_ld(uint32_t ta, float (&v)[NC]) {
  const int lane0 = (int)(ta >> 16), col = (int)(ta & 0xffff);
  if (lane0 != 32 * (int)((threadIdx.x >> 5) & 3)) emu_fail("load outside the warp's lane quarter");
  if (col + NC > 512) emu_fail("load outside tensor memory");
  __syncwarp();
  for (int i = 0; i < NC; ++i) v[i] = emu_tc()->tmem[lane0 + (threadIdx.x & 31)][col + i];
  __syncwarp();
}
inline void ld32(uint32_t ta, float (&v)[32]) { emu_ld<32>(ta, v); }
inline void ld32_raw(uint32_t ta, uint32_t (&r)[32]) {
  float v[32];
  emu_ld<32>(ta, v);
  memcpy(r, v, sizeof(v));
}
inline void wait_ld(uint32_t (&)[32]) {}
inline void ld16(uint32_t ta, float (&v)[16]) { emu_ld<16>(ta, v); }

}  // namespace tc
}  // namespace vio
