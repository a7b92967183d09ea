"""Writes tests/golden/fpr_closed_form.json from the oracle only.

Closed-form expected FPR (ideal hashing) for the workload geometries: the
1 MiB filter with 10^6 keys, and the 32 MiB / 4 GiB filters at 10 bits per
key for every valid (B, S, k) with B in {128, 256, 512}, S in {32, 64} and
k in {4, 8, 16}.  Run from the repository root:

    python tests/golden/gen_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402


def main():
    rows = []
    rows.append(dict(name="1MiB_n1e6", num_blocks=1 << 15, n=10**6, block_bits=256, word_bits=32, k=8))
    rows.append(dict(name="1MiB_n2^20", num_blocks=1 << 15, n=1 << 20, block_bits=256, word_bits=32, k=8))
    for size_name, nbytes in (("32MiB", 32 << 20), ("4GiB", 4 << 30)):
        for B in (128, 256, 512):
            for S in (32, 64):
                for k in (4, 8, 16):
                    s = B // S
                    if k < s or k % s:
                        continue
                    b = nbytes * 8 // B
                    n = nbytes * 8 // 10
                    rows.append(dict(name=f"{size_name}_B{B}_S{S}_k{k}", num_blocks=b, n=n,
                                     block_bits=B, word_bits=S, k=k))
    for r in rows:
        r["fpr"] = oracle.fpr_sbf_closed_form(r["num_blocks"], r["n"], r["block_bits"], r["word_bits"], r["k"])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fpr_closed_form.json")
    with open(out, "w") as f:
        json.dump({"source": "oracle.fpr_sbf_closed_form (ideal hashing, exact)", "rows": rows}, f, indent=1)
    print(f"wrote {len(rows)} rows to {out}")


if __name__ == "__main__":
    main()
