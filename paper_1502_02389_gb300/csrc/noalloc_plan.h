// Launch planning of lift_asum_noalloc, in plain C++ with no CUDA
// dependency, so that the argument path (which loads the full tiles use, how
// many CTAs and partial slots a call needs, which arguments are refused) can
// be checked on a machine without a GPU.  noalloc.cu calls it before every
// launch; a host-only test compiles it on its own.
#pragma once
#include <stdint.h>

namespace lift {
namespace noalloc {

constexpr int kSlots = 4096;    // partial slots of the fixed scratch array
constexpr int kThreads = 256;   // threads per CTA
constexpr int kTile = 4096;     // elements per CTA tile (split^4096)
constexpr int kVW = 4;          // elements per thread load (asVector^4)

enum Result { kOk = 0, kBadArgs = 1, kTooLarge = 2, kNoResidentCta = 3 };

struct Plan {
  int64_t grid = 0;        // CTAs of the launch, one partial slot each
  bool vector_loads = false;  // full tiles read with 16-byte loads (x 16-byte aligned)
};

// x: the input (device address, only its value is inspected); n: elements;
// sms: SMs of the device; per_sm: CTAs of the kernel resident per SM.
inline Result plan(const void* x, int64_t n, bool have_result, int sms, int per_sm, Plan* out) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(x);
  if (n < 0 || !have_result || (n > 0 && !x) || a % 4 != 0) return kBadArgs;
  if (sms < 1 || per_sm < 1) return kNoResidentCta;
  const int64_t tiles = n > 0 ? (n + kTile - 1) / kTile : 1;
  const int64_t cap = (int64_t)sms * per_sm;
  out->grid = tiles < cap ? tiles : cap;
  // 16-byte vector loads need a 16-byte aligned x (then every full tile's
  // vector starts are too: a tile is 16 KiB, a vector 16 bytes); a 4-byte
  // aligned x is read element by element in the same order
  out->vector_loads = a % 16 == 0;
  if (out->grid > kSlots) return kTooLarge;
  return kOk;
}

}  // namespace noalloc
}  // namespace lift
