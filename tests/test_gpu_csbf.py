"""Cache-sectorized filters (Sec. II-A, CSBF) on the GPU against the oracle:
bit array and every answer identical, for every compiled (B, S, K, z) and
every layout, on ragged sizes."""
import numpy as np
import pytest

import oracle
import synthkeys
from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GEOMETRIES = [(64, 32), (128, 32), (256, 32), (512, 32), (64, 64), (128, 64), (256, 64), (512, 64), (1024, 64)]


def compiled_csbf():
    for B, S in GEOMETRIES:
        s = B // S
        for z in (1, 2, 4, 8):
            if z >= s:
                continue
            for k in (4, 8, 16):
                if k % z == 0:
                    yield B, S, k, z


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2512_15595_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("B,S,k,z", list(compiled_csbf()))
def test_csbf_every_layout_bit_exact(torch, B, S, k, z):
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, Filter
    geom = oracle.Geometry(num_blocks=1013, block_bits=B, word_bits=S, k=k, seed=0x5EED, groups=z)
    n = 1013 * B // 16 + 9
    ins = synthkeys.insert_keys(n, seed=12)
    q, _ = synthkeys.mixed_queries(n, 1000, 2001, seed_insert=12)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    dk = torch.from_numpy(ins.view(np.int64)).cuda()
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    cg = 1
    while cg <= z:
        for kpt in (1, 2, 4):
            f = Filter(geom.num_blocks, B, S, k, geom.seed, groups=z)
            f.set_layout(BF_OP_ADD, cg=cg, phi=1, kpt=kpt)
            f.set_layout(BF_OP_CONTAINS, cg=cg, phi=1, kpt=kpt)
            f.add(dk)
            out = f.contains(dq)
            assert np.array_equal(f.words.cpu().numpy(), ref.as_bytes()), (cg, kpt)
            assert np.array_equal(out.cpu().numpy().astype(np.uint8), ref_out), (cg, kpt)
            f.close()
        cg *= 2


def test_csbf_with_one_word_per_group_is_the_sbf(torch):
    from paper_2512_15595_gb300 import Filter
    ins = torch.from_numpy(synthkeys.insert_keys(50_000).view(np.int64)).cuda()
    a = Filter(4099, 512, 64, 16, 3, groups=8)
    b = Filter(4099, 512, 64, 16, 3)
    a.add(ins)
    b.add(ins)
    assert torch.equal(a.words, b.words)
