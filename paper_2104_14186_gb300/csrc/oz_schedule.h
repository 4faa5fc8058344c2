// Host-side schedule of the emulated-FP64 digit products (ozaki.cu): which digit tiles each
// K step loads, which tensor-memory accumulator ("slot") each digit pair adds into, and when a
// slot is flushed into the FP64 sums.  Plain C++ (no CUDA), so that it can be checked on the
// host against exact arithmetic.
//
// Digit pairs (s, t) with s + t <= kOzT, s, t in [1, kOzS], are grouped into 2 x 2 blocks
// anchored at odd (s0, t0): the block loads op(A) digits s0, s0 + 1 and op(B) digits t0,
// t0 + 1 once per K step and runs up to four pair products from them (66 digit tiles per K
// step for the 60 pairs, instead of 120 when every pair loads its own two).  A block touches
// the levels s0 + t0, s0 + t0 + 1 (two pairs) and s0 + t0 + 2; pairs of one level share a slot,
// whose FP32 sums stay exact while it holds at most kOzSlotBudget pair-steps.  Blocks run in
// order of their anchor level, so a level's slot carries over from one block to the next; a
// slot is flushed when its level is done or its budget would overflow, and reused once the
// flush has drained it.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define QDWHP_OZ_HD __host__ __device__
#else
#define QDWHP_OZ_HD
#endif

namespace qdwhp {

constexpr int kOzS = 9;              // digits per entry
constexpr int kOzT = 12;             // keep digit pairs with s + t <= kOzT (1-based)
constexpr int kOzStepK = 64;         // K per step (one 128-byte swizzle atom of bfloat16)
constexpr int kOzChunk = 128;        // K steps per schedule item at most (8192 deep): two pairs of one
                                     // level over a whole item fill a slot's budget
constexpr int kOzSlots = 4;          // 128-column FP32 accumulators in tensor memory
constexpr int kOzSlotBudget = 256;   // pair-steps per slot between flushes: 256 x 64 digit products of
                                     // magnitude <= 2^10 keep every partial sum <= 2^24 (exact in FP32)
constexpr int kOzMaxItems = 320;
constexpr int kOzMaxFlush = 640;
constexpr int kOzMaxSteps = 8 * kOzChunk;   // K steps per launch at most (65536 deep); longer K is split

// One launch's schedule, passed by value as a kernel parameter (3.2 KB).
struct OzSchedule {
  int nitems, nflush, nsteps, clen;   // clen: K steps per item (the last item of a block may have fewer)
  uint8_t atile[kOzMaxItems];    // op(A) digit of tile 0 | digit of tile 1 << 4 (0-based; 0xF: none)
  uint8_t btile[kOzMaxItems];    // op(B) digits likewise
  uint8_t pair[kOzMaxItems][4];  // bit 7 valid; bit 0 A tile; bit 1 B tile; bits 2-3 slot; bit 4 the
                                 // pair's first product overwrites the slot (first step of the item)
  uint8_t chunk[kOzMaxItems];    // K steps [chunk * clen, min(chunk * clen + clen, nsteps))
  uint8_t ctl[kOzMaxItems];      // bits 0-3: slots whose last flush must have drained before the
                                 // item's first step; bits 4-6: flushes issued after the item
  uint8_t flush[kOzMaxFlush];    // slot | level << 2, in issue order
};

// kernel parameters are limited to 4 KB on the classic path; the two tensor maps and the
// scalars take about 0.4 KB of it
static_assert(sizeof(OzSchedule) <= 3584, "the digit-pair schedule must fit in a kernel parameter block");

QDWHP_OZ_HD inline int oz_item_steps(const OzSchedule& s, int it) {
  const int left = s.nsteps - s.chunk[it] * s.clen;
  return left < s.clen ? left : s.clen;
}

// Builds the schedule for nsteps K steps (1 <= nsteps <= kOzMaxSteps).  false if it would not fit.
inline bool oz_build_schedule(int nsteps, OzSchedule* out) {
  if (nsteps < 1 || nsteps > kOzMaxSteps) return false;
  OzSchedule& S = *out;
  std::memset(&S, 0, sizeof(S));
  S.nsteps = nsteps;
  const int nchunks = (nsteps + kOzChunk - 1) / kOzChunk;
  S.clen = (nsteps + nchunks - 1) / nchunks;   // balanced chunks of at most kOzChunk steps
  // blocks in anchor-level order; pairs of a block listed (s0,t0), (s0,t0+1), (s0+1,t0), (s0+1,t0+1)
  struct Blk {
    int a[2], b[2], na, nb, np, ps[4], pt[4];
  };
  Blk blk[32];
  int nblk = 0;
  for (int L = 2; L <= kOzT; L += 2)
    for (int s0 = 1; s0 <= kOzS; s0 += 2) {
      const int t0 = L - s0;
      if (t0 < 1 || t0 > kOzS) continue;
      Blk b{};
      b.a[0] = s0;
      b.b[0] = t0;
      b.na = b.nb = 1;
      for (int ds = 0; ds < 2; ++ds)
        for (int dt = 0; dt < 2; ++dt) {
          const int s = s0 + ds, t = t0 + dt;
          if (s > kOzS || t > kOzS || s + t > kOzT) continue;
          if (ds) { b.a[1] = s; b.na = 2; }
          if (dt) { b.b[1] = t; b.nb = 2; }
          b.ps[b.np] = s;
          b.pt[b.np] = t;
          ++b.np;
        }
      blk[nblk++] = b;
    }
  const int nitems = nblk * nchunks;
  if (nitems > kOzMaxItems) return false;
  S.nitems = nitems;
  // last item that uses each level
  int last_use[kOzT + 1];
  for (int l = 0; l <= kOzT; ++l) last_use[l] = -1;
  for (int bi = 0; bi < nblk; ++bi)
    for (int p = 0; p < blk[bi].np; ++p) last_use[blk[bi].ps[p] + blk[bi].pt[p]] = bi * nchunks + nchunks - 1;
  int lvl[kOzSlots], used[kOzSlots], nfl[kOzSlots], lastfl[kOzSlots];
  for (int x = 0; x < kOzSlots; ++x) { lvl[x] = -1; used[x] = 0; nfl[x] = 0; lastfl[x] = -1000000; }
  int nflush = 0;
  auto emit_flush = [&](int after_item, int x) -> bool {
    if (nflush >= kOzMaxFlush || after_item < 0 || nfl[x] >= 255) return false;   // 8-bit counters in the kernel
    const int cnt = (S.ctl[after_item] >> 4) & 7;
    if (cnt >= 7) return false;
    S.ctl[after_item] = (uint8_t)((S.ctl[after_item] & 0x0F) | ((cnt + 1) << 4));
    S.flush[nflush++] = (uint8_t)(x | (lvl[x] << 2));
    ++nfl[x];
    lastfl[x] = after_item;
    lvl[x] = -1;
    used[x] = 0;
    return true;
  };
  for (int bi = 0; bi < nblk; ++bi)
    for (int c = 0; c < nchunks; ++c) {
      const int it = bi * nchunks + c;
      const Blk& b = blk[bi];
      S.chunk[it] = (uint8_t)c;
      const int len = oz_item_steps(S, it);
      S.atile[it] = (uint8_t)((b.a[0] - 1) | ((b.na == 2 ? b.a[1] - 1 : 0xF) << 4));
      S.btile[it] = (uint8_t)((b.b[0] - 1) | ((b.nb == 2 ? b.b[1] - 1 : 0xF) << 4));
      bool seen[kOzT + 2] = {};
      for (int p = 0; p < b.np; ++p) {
        const int L = b.ps[p] + b.pt[p];
        int x = -1;
        for (int y = 0; y < kOzSlots; ++y)
          if (lvl[y] == L) x = y;
        bool fresh = false;
        if (!seen[L]) {
          int need = 0;
          for (int q = 0; q < b.np; ++q)
            if (b.ps[q] + b.pt[q] == L) need += len;
          if (x >= 0 && used[x] + need > kOzSlotBudget) {
            if (!emit_flush(it - 1, x)) return false;
            x = -1;
          }
          if (x < 0) {
            // the free slot flushed longest ago (its drain is the most likely to be done)
            for (int y = 0; y < kOzSlots; ++y)
              if (lvl[y] == -1 && (x < 0 || lastfl[y] < lastfl[x])) x = y;
            if (x < 0) return false;   // cannot happen: a block touches at most 3 levels
            lvl[x] = L;
            used[x] = 0;
            fresh = true;
            if (nfl[x] > 0) S.ctl[it] |= (uint8_t)(1u << x);
          }
          used[x] += need;
          seen[L] = true;
        }
        const int ai = b.ps[p] == b.a[0] ? 0 : 1, bti = b.pt[p] == b.b[0] ? 0 : 1;
        S.pair[it][p] = (uint8_t)(0x80 | ai | (bti << 1) | (x << 2) | (fresh ? 0x10 : 0));
      }
      for (int x = 0; x < kOzSlots; ++x)
        if (lvl[x] != -1 && last_use[lvl[x]] == it && !emit_flush(it, x)) return false;
    }
  S.nflush = nflush;
  return true;
}

}  // namespace qdwhp
