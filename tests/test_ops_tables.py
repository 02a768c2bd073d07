"""The FP32 operator tables compiled into the FMA stage kernel
(csrc/ops_tables.inc) equal the library's runtime operators rounded to FP32,
bit for bit, for degrees 0..5 (a stale table would change the kernel's
Dr, Ds and LIFT without any other sign)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2012_13487_gb300", "csrc", "ops_tables.inc")


def parse_tables():
    text = open(INC).read()
    out = {}
    for m in re.finditer(r"#(?:el)?if FEDBM_P == (\d+)\n#define FEDBM_OPS32_TABLE \\\n(.*?)(?=\n#)", text, re.S):
        vals = re.findall(r"(-?0x[0-9a-f.]+p[+-]\d+)f", m.group(2))
        out[int(m.group(1))] = np.array([float.fromhex(v) for v in vals], dtype=np.float32)
    return out


@pytest.mark.parametrize("p", range(6))
def test_ops_table_matches_runtime_operators(p):
    from paper_2012_13487_gb300 import fedbm as fb
    o = fb.fedbm_ref_operators(p)
    want = np.concatenate([o["Dr"].ravel(), o["Ds"].ravel(), o["LIFT"].ravel()]).astype(np.float32)
    got = parse_tables()[p]
    assert got.shape == want.shape
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
