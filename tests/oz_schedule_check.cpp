// Host check of the emulated-FP64 digit-pair schedule (paper_2104_14186_gb300/csrc/oz_schedule.h),
// run by tests/test_oz_schedule.py.  For one output entry it plays the schedule the way the
// product kernel reads it: per item and K step, every valid pair product added into its slot
// (FP32, beside an exact int64 shadow), the "fresh" pairs overwriting their slot on the item's
// first step, and after each item the listed flushes added into an FP64 sum times 2^(-6 level).
// It fails on:
//   * a pair covered other than once per K step, or a kept pair (s + t <= 12) missed;
//   * an FP32 partial sum that differs from the exact one, or above 2^24 in magnitude;
//   * a slot read by a pair of another level, a flush of the wrong level, a slot never flushed;
//   * a reused slot without the wait bit;
//   * a final FP64 sum off the exact digit sum by more than the FP64 rounding of its flushes.
// Digits are random in [-32, 32], or all 32 (every product at the 2^10 bound, same sign).
// Usage: oz_schedule_check  (prints "ok" and exits 0, else prints the failure and exits 1)
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "oz_schedule.h"

using namespace qdwhp;

static int check(int nsteps, int mode, unsigned seed) {
  OzSchedule S;
  if (!oz_build_schedule(nsteps, &S)) {
    std::printf("no schedule for %d steps\n", nsteps);
    return 1;
  }
  const int K = nsteps * kOzStepK;
  std::mt19937 g(seed);
  std::vector<int> DA((size_t)kOzS * K), DB((size_t)kOzS * K);
  for (auto& d : DA) d = mode == 0 ? 32 : (int)(g() % 65) - 32;
  for (auto& d : DB) d = mode == 0 ? 32 : (int)(g() % 65) - 32;
  // exact value: sum over levels L of 2^(-6 L) S_L, S_L an integer
  long long SL[kOzT + 1] = {};
  for (int s = 1; s <= kOzS; ++s)
    for (int t = 1; t <= kOzS; ++t) {
      if (s + t > kOzT) continue;
      long long acc = 0;
      for (int k = 0; k < K; ++k) acc += (long long)DA[(size_t)(s - 1) * K + k] * DB[(size_t)(t - 1) * K + k];
      SL[s + t] += acc;
    }
  long double exact = 0, scale = 0;
  for (int L = 2; L <= kOzT; ++L) {
    exact += std::ldexp((long double)SL[L], -6 * L);
    scale += std::ldexp(std::fabs((long double)SL[L]), -6 * L);
  }
  float slot[kOzSlots] = {};
  long long shadow[kOzSlots] = {};
  int lev[kOzSlots], flushed[kOzSlots] = {};
  for (int x = 0; x < kOzSlots; ++x) lev[x] = -1;
  std::vector<int> cover((size_t)kOzS * kOzS * nsteps, 0);
  double acc64 = 0;
  int fp = 0;
  for (int it = 0; it < S.nitems; ++it) {
    const int k0 = S.chunk[it] * S.clen, len = oz_item_steps(S, it);
    const int a[2] = {S.atile[it] & 15, S.atile[it] >> 4}, b[2] = {S.btile[it] & 15, S.btile[it] >> 4};
    for (int p = 0; p < 4; ++p) {
      const int c = S.pair[it][p];
      const int x = (c >> 2) & 3;
      if ((c & 0x80) && (c & 0x10) && flushed[x] > 0 && !((S.ctl[it] >> x) & 1)) {
        std::printf("item %d reuses slot %d without waiting for its flush\n", it, x);
        return 1;
      }
    }
    for (int st = 0; st < len; ++st) {
      const int kb = k0 + st;
      for (int p = 0; p < 4; ++p) {
        const int c = S.pair[it][p];
        if (!(c & 0x80)) continue;
        const int s = a[c & 1], t = b[(c >> 1) & 1], x = (c >> 2) & 3;
        if (s == 15 || t == 15 || s + t + 2 > kOzT) {
          std::printf("item %d: pair outside the kept set\n", it);
          return 1;
        }
        const int L = s + t + 2;
        if ((c & 0x10) && st == 0) {
          slot[x] = 0.0f;
          shadow[x] = 0;
          lev[x] = L;
        }
        if (lev[x] != L) {
          std::printf("item %d: slot %d holds level %d, pair level %d\n", it, x, lev[x], L);
          return 1;
        }
        cover[((size_t)s * kOzS + t) * nsteps + kb]++;
        for (int kk = 0; kk < kOzStepK; ++kk) {
          const size_t k = (size_t)kb * kOzStepK + kk;
          const long long pr = (long long)DA[(size_t)s * K + k] * DB[(size_t)t * K + k];
          shadow[x] += pr;
          slot[x] += (float)pr;
          if (std::llabs(shadow[x]) > (1LL << 24) || (long long)slot[x] != shadow[x]) {
            std::printf("item %d slot %d: FP32 sum not exact (%lld)\n", it, x, shadow[x]);
            return 1;
          }
        }
      }
    }
    const int nf = (S.ctl[it] >> 4) & 7;
    for (int f = 0; f < nf; ++f) {
      const int fl = S.flush[fp++], x = fl & 3, L = fl >> 2;
      if (lev[x] != L) {
        std::printf("flush of slot %d at level %d, slot holds %d\n", x, L, lev[x]);
        return 1;
      }
      acc64 += std::ldexp((double)slot[x], -6 * L);
      lev[x] = -1;
      ++flushed[x];
    }
  }
  if (fp != S.nflush) {
    std::printf("%d flushes issued, %d listed\n", fp, S.nflush);
    return 1;
  }
  for (int x = 0; x < kOzSlots; ++x)
    if (lev[x] != -1) {
      std::printf("slot %d never flushed\n", x);
      return 1;
    }
  for (int s = 0; s < kOzS; ++s)
    for (int t = 0; t < kOzS; ++t)
      for (int kb = 0; kb < nsteps; ++kb) {
        const int want = (s + t + 2 <= kOzT) ? 1 : 0;
        if (cover[((size_t)s * kOzS + t) * nsteps + kb] != want) {
          std::printf("pair (%d,%d) step %d covered %d times\n", s + 1, t + 1, kb,
                      cover[((size_t)s * kOzS + t) * nsteps + kb]);
          return 1;
        }
      }
  // each flush adds one FP64 rounding of at most 2^-53 of the running magnitude
  const long double bound = (long double)(S.nflush + 1) * std::ldexp(1.0L, -53) * scale;
  if (std::fabs((long double)acc64 - exact) > bound) {
    std::printf("steps %d: FP64 sum off by %Lg (bound %Lg)\n", nsteps, std::fabs((long double)acc64 - exact), bound);
    return 1;
  }
  return 0;
}

int main() {
  const int ns[] = {1, 2, 3, 5, 16, 63, 64, 65, 100, 127, 128, 129, 200, 256, 257, 300, 383, 511, 512, 700, 1023,
                    kOzMaxSteps};
  for (int n : ns)
    for (int mode = 0; mode < 2; ++mode)
      for (unsigned seed = 1; seed <= 2; ++seed)
        if (check(n, mode, seed)) return 1;
  OzSchedule S;
  if (oz_build_schedule(kOzMaxSteps + 1, &S) || oz_build_schedule(0, &S)) {
    std::printf("a schedule outside [1, kOzMaxSteps] steps was built\n");
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
