// Host-only check of lift_asum_noalloc's launch planning (the header the
// entry point calls before every launch): which loads a call's full tiles
// use, its grid, and the arguments it refuses -- all decided before any
// CUDA call.  Prints one line per case; exits non-zero on a mismatch.
#include <stdio.h>

#include "noalloc_plan.h"

using namespace lift::noalloc;

static int failures = 0;

static void expect(const char* what, bool ok) {
  printf("%s %s\n", ok ? "ok  " : "FAIL", what);
  if (!ok) ++failures;
}

int main() {
  alignas(16) static float buf[64];
  const char* base = reinterpret_cast<const char*>(buf);
  Plan p;
  // 16-byte aligned x: vector loads
  expect("aligned x plans vector loads",
         plan(base, 1 << 20, true, 152, 8, &p) == kOk && p.vector_loads && p.grid == 256);
  // x offset by 1, 2, 3 floats: 4-byte loads, same grid
  for (int off = 1; off <= 3; ++off) {
    const bool ok = plan(base + 4 * off, (1 << 20) + 7, true, 152, 8, &p) == kOk &&
                    !p.vector_loads && p.grid == 257;
    expect("4-byte aligned x plans scalar loads", ok);
  }
  expect("x offset by 8 bytes plans scalar loads",
         plan(base + 8, 5000, true, 152, 8, &p) == kOk && !p.vector_loads && p.grid == 2);
  // arguments refused before any launch
  expect("x not 4-byte aligned refused", plan(base + 2, 100, true, 152, 8, &p) == kBadArgs);
  expect("n < 0 refused", plan(base, -1, true, 152, 8, &p) == kBadArgs);
  expect("NULL x with n > 0 refused", plan(nullptr, 5, true, 152, 8, &p) == kBadArgs);
  expect("NULL result refused", plan(base, 5, false, 152, 8, &p) == kBadArgs);
  expect("NULL x with n == 0 accepted, one CTA",
         plan(nullptr, 0, true, 152, 8, &p) == kOk && p.grid == 1);
  // grid: min(tiles, SMs x resident CTAs); beyond the scratch array: refused
  expect("grid capped at SMs x CTAs per SM",
         plan(base, int64_t(1) << 31, true, 152, 8, &p) == kOk && p.grid == 1216);
  expect("grid beyond 4096 slots refused",
         plan(base, int64_t(1) << 31, true, 600, 8, &p) == kTooLarge);
  expect("no resident CTA reported as such", plan(base, 100, true, 152, 0, &p) == kNoResidentCta);
  printf(failures ? "failed\n" : "all ok\n");
  return failures ? 1 : 0;
}
