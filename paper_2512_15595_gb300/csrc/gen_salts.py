"""Writes salts.cuh: the multiplier tables the kernels inline as literals.

Salt i of the 64-bit table is the i-th output (i = 0..63) of a SplitMix64
generator seeded with 0x5A175EED, with the low bit forced to 1 (the
multipliers must be odd, Sec. IV-B).  Salt i of the 32-bit table is
(salt64_i >> 32) | 1.  Run from this directory:  python gen_salts.py
"""
import os

SEED = 0x5A175EED
M = (1 << 64) - 1


def table64(count=64):
    state, out = SEED, []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append((z ^ (z >> 31)) | 1)
    return out


def main():
    t64 = table64()
    t32 = [((x >> 32) | 1) & 0xFFFFFFFF for x in t64]
    lines = [
        "// Generated by gen_salts.py -- do not edit.",
        "// Odd multipliers for the salted multiplicative bit positions (Sec. IV-B).",
        "// salt64[i] = SplitMix64(seed 0x5A175EED) output i, low bit set;",
        "// salt32[i] = (salt64[i] >> 32) | 1.",
        "#pragma once",
        "#include <cstdint>",
        "namespace bloomgb {",
        "constexpr int kMaxSalts = 64;",
        "__host__ __device__ constexpr uint64_t salt64_at(int i) {",
        "  switch (i) {",
    ]
    lines += [f"    case {i}: return 0x{v:016X}ull;" for i, v in enumerate(t64)]
    lines += ["    default: return 0;", "  }", "}",
              "__host__ __device__ constexpr uint32_t salt32_at(int i) {", "  switch (i) {"]
    lines += [f"    case {i}: return 0x{v:08X}u;" for i, v in enumerate(t32)]
    lines += ["    default: return 0;", "  }", "}", "}  // namespace bloomgb", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "salts.cuh")
    with open(out, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
