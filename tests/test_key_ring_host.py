"""The lookup server's key arena (csrc/key_ring.h) on the CPU: random
admission / completion sequences, shaped like the server's (several runs per
launch, launches completed in order, empty requests), against a model that
tracks every live run.  Checked after every step: a run lies inside the
ring and overlaps no live run; the ring's count of used slots equals the
model's; a request that fits an empty ring is always admitted; an empty
request consumes nothing.  Host logic only (g++, no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <deque>
#include <vector>
#include "key_ring.h"

struct Run { uint64_t off, n; };
struct Group { std::vector<Run> runs; uint64_t consumed = 0, end = 0; };

static uint64_t st;
static uint64_t rnd() {  // SplitMix64
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int main(int argc, char** argv) {
  const uint64_t cap = std::strtoull(argv[1], nullptr, 10);
  st = std::strtoull(argv[2], nullptr, 10);
  const int steps = std::atoi(argv[3]);
  bloomgb::KeyRing ring;
  ring.cap = cap;
  std::deque<Group> live;
  uint64_t takes = 0, wraps = 0, refusals = 0;
  for (int t = 0; t < steps; ++t) {
    if (!live.empty() && (rnd() % 3 == 0)) {  // complete the oldest launch
      ring.release(live.front().consumed, live.front().end);
      live.pop_front();
    } else {  // admit a launch of up to 4 requests, stopping at the first that does not fit
      Group g;
      const int nreq = 1 + rnd() % 4;
      for (int r = 0; r < nreq; ++r) {
        const uint64_t kind = rnd() % 8;
        const uint64_t n = kind == 0 ? 0 : (kind == 1 ? cap : 1 + rnd() % (cap / 3 + 1));
        uint64_t off = 0, consumed = 0;
        const bool empty_ring = ring.used == 0;
        if (!ring.take(n, &off, &consumed)) {
          if (empty_ring && n <= cap && g.runs.empty()) { std::printf("FAIL refused %llu on an empty ring\n", (unsigned long long)n); return 1; }
          ++refusals;
          break;
        }
        ++takes;
        if (n == 0) {
          if (consumed != 0) { std::printf("FAIL empty request consumed %llu\n", (unsigned long long)consumed); return 1; }
          continue;
        }
        if (consumed != n) ++wraps;
        if (off + n > cap) { std::printf("FAIL run [%llu,+%llu) outside the ring\n", (unsigned long long)off, (unsigned long long)n); return 1; }
        for (const Group& h : live)
          for (const Run& x : h.runs)
            if (off < x.off + x.n && x.off < off + n) { std::printf("FAIL overlap with a live run\n"); return 1; }
        for (const Run& x : g.runs)
          if (off < x.off + x.n && x.off < off + n) { std::printf("FAIL overlap within a launch\n"); return 1; }
        g.runs.push_back({off, n});
        g.consumed += consumed;
      }
      g.end = ring.head;
      live.push_back(g);
    }
    uint64_t used = 0;
    for (const Group& h : live) used += h.consumed;
    if (used != ring.used) { std::printf("FAIL used %llu, model %llu\n", (unsigned long long)ring.used, (unsigned long long)used); return 1; }
    if (ring.used > cap) { std::printf("FAIL used beyond capacity\n"); return 1; }
  }
  while (!live.empty()) { ring.release(live.front().consumed, live.front().end); live.pop_front(); }
  if (ring.used || ring.head || ring.tail) { std::printf("FAIL not empty after releasing everything\n"); return 1; }
  std::printf("ok %llu %llu %llu\n", (unsigned long long)takes, (unsigned long long)wraps, (unsigned long long)refusals);
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("ring")
    src = d / "ring.cpp"
    src.write_text(HARNESS)
    exe = d / "ring"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2512_15595_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    return exe


@pytest.mark.parametrize("cap", [1, 2, 7, 64, 1000, 4096])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_key_ring_random_sequences(harness, cap, seed):
    p = subprocess.run([str(harness), str(cap), str(seed), "20000"], capture_output=True, text=True)
    assert p.returncode == 0, p.stdout
    _, takes, wraps, refusals = p.stdout.split()
    assert int(takes) > 1000
    if cap >= 7:
        assert int(refusals) > 0  # the full-ring path ran
    if cap >= 64:
        assert int(wraps) > 0  # and the wrap to slot 0
