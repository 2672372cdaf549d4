// Scratch arithmetic of the allocation-free solve (dj_sssp_noalloc).  Plain
// host C++ with no CUDA header, so that a host-only test can check the limits
// the documentation states against the size of the fixed array.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>

namespace dj {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // the fixed device array: 4 MiB
constexpr size_t kNoAllocCtlBytes = 256;                   // barrier and candidate counters (zeroed per call)
constexpr size_t kNoAllocWordBytes = 64;                   // error bits and phase count (zeroed per call)
constexpr int kNoAllocMaxCtas = 320;                       // the grid engine's decision warp reads <= 320 partials
constexpr size_t kNoAllocEntryBytes = 16;                  // one partial or one published candidate (a uint4)

// CTAs of the grid engine on a matrix of row pitch `pitch` (a multiple of 32)
// with `num_sms` SMs, one CTA per SM.
inline int noalloc_ctas(int32_t pitch, int num_sms) {
  return std::max(1, std::min({num_sms, static_cast<int>(pitch / 4), kNoAllocMaxCtas}));
}

// Columns of the widest CTA slice (a multiple of 4).
inline int noalloc_slice_cap(int32_t pitch, int num_sms) {
  const int nvec_total = static_cast<int>(pitch / 4);
  const int G = noalloc_ctas(pitch, num_sms);
  return 4 * std::max(1, (nvec_total + G - 1) / G);
}

// Bytes the solve needs: counters, status words, two phase-parity copies of
// the G per-CTA partials, and two copies of the G candidate regions of one
// slice each -- about 2 * 16 * pitch bytes, i.e. 32 bytes per column.
inline size_t noalloc_scratch_bytes(int32_t pitch, int num_sms) {
  const size_t G = static_cast<size_t>(noalloc_ctas(pitch, num_sms));
  const size_t swcap = static_cast<size_t>(noalloc_slice_cap(pitch, num_sms));
  return kNoAllocCtlBytes + kNoAllocWordBytes + 2 * G * kNoAllocEntryBytes + 2 * G * swcap * kNoAllocEntryBytes;
}

// The largest row pitch (so the largest n, pitch being n rounded up to 32)
// whose scratch fits the fixed array on a device with `num_sms` SMs.
inline int32_t noalloc_max_pitch(int num_sms) {
  int32_t lo = 32, hi = 32;
  while (noalloc_scratch_bytes(hi * 2, num_sms) <= kNoAllocScratchBytes && hi < (1 << 29)) hi *= 2;
  hi *= 2;  // scratch(hi) > limit, scratch(lo) <= limit (monotone in the pitch)
  while (hi - lo > 32) {
    const int32_t mid = lo + ((hi - lo) / 64) * 32;
    if (noalloc_scratch_bytes(mid, num_sms) <= kNoAllocScratchBytes)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

}  // namespace dj
