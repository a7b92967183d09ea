"""The multipliers are a project convention (the paper gives none, Sec. IV-B).
Both sides generate them on their own: the CUDA side's table is literal text in
csrc/salts.cuh (written by csrc/gen_salts.py), the oracle's comes from its own
SplitMix64 in C.  The two tables must be identical."""
import os
import re

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2512_15595_gb300", "csrc", "salts.cuh")


def parse(fn_name):
    text = open(HDR).read()
    body = text[text.index(fn_name):]
    body = body[: body.index("default:")]
    return {int(i): int(v, 16) for i, v in re.findall(r"case (\d+): return 0x([0-9A-Fa-f]+)", body)}


def test_salt64_table_matches_oracle():
    t = parse("salt64_at")
    assert sorted(t) == list(range(64))
    assert [t[i] for i in range(64)] == oracle.salts(64)


def test_salt32_table_matches_oracle():
    t = parse("salt32_at")
    assert sorted(t) == list(range(64))
    assert [t[i] for i in range(64)] == oracle.salts(32)


def test_parquet_salt_table_matches_oracle():
    """The CUDA side's Parquet split-block multipliers (csrc/parquet_salts.cuh)
    equal the oracle's, which the pyarrow pins tie to the Parquet writer."""
    text = open(os.path.join(ROOT, "paper_2512_15595_gb300", "csrc", "parquet_salts.cuh")).read()
    body = text[text.index("parquet_salt32_at"):]
    body = body[: body.index("default:")]
    t = {int(i): int(v, 16) for i, v in re.findall(r"case (\d+): return 0x([0-9A-Fa-f]+)", body)}
    assert sorted(t) == list(range(8))
    assert [t[i] for i in range(8)] == oracle.parquet_salts()
