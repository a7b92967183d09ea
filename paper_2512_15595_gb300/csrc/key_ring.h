// Key arena of the lookup server: a ring of `cap` key slots handed out in
// contiguous runs and released in the order they were taken.  Host-only
// logic (no CUDA), shared by the server and its CPU test.
#pragma once

#include <algorithm>
#include <cstdint>

namespace bloomgb {

struct KeyRing {
  uint64_t cap = 0;   // slots
  uint64_t head = 0;  // next slot to hand out
  uint64_t tail = 0;  // first slot still in use (occupied: [tail, head) mod cap)
  uint64_t used = 0;  // occupied slots, including ends skipped by a wrap

  // Take n slots as one contiguous run, wrapping to slot 0 when the end of
  // the ring is too short (the skipped end is consumed by this run until it
  // is released).  Returns false if there is no room now; else the run's
  // first slot in *off and the slots it consumed in *consumed (0 for n = 0).
  bool take(uint64_t n, uint64_t* off, uint64_t* consumed) {
    if (n > cap) return false;
    if (n == 0) {
      *off = head < cap ? head : 0;
      *consumed = 0;
      return true;
    }
    if (used == 0) head = tail = 0;
    if (used >= cap) return false;
    if (used == 0 || head > tail) {
      // free: [head, cap) and [0, tail)
      if (cap - head >= n) {
        *off = head;
        *consumed = n;
        head += n;
        used += n;
        return true;
      }
      if (tail >= n) {
        *consumed = (cap - head) + n;
        used += *consumed;
        *off = 0;
        head = n;
        return true;
      }
      return false;
    }
    // head < tail: free is [head, tail)
    if (tail - head >= n) {
      *off = head;
      *consumed = n;
      head += n;
      used += n;
      return true;
    }
    return false;
  }

  // Release the slots of the oldest outstanding group of runs: `consumed`
  // slots ending at ring position `end` (the head right after the group was
  // taken).  A group that consumed nothing releases nothing.
  void release(uint64_t consumed, uint64_t end) {
    if (consumed == 0) return;
    used -= std::min(used, consumed);
    tail = end;
    if (used == 0) head = tail = 0;
  }
};

}  // namespace bloomgb
