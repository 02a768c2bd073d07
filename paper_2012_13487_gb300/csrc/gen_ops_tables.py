"""Writes ops_tables.inc: the FP32 Dr, Ds and LIFT operators of degrees 0..5
as compile-time tables for the FMA stage kernel.

The nodal Lagrange basis of Sec. II.B.1 lives on one reference triangle, so
Dr, Ds and LIFT depend only on the degree (and on the node set, which the paper
leaves open: warp & blend nodes with alpha = 0 here).  The FP32 kernels can
therefore take them as instruction immediates instead of loading them from
constant memory.  The values are the library's own operators
(``fedbm_ref_operators``) rounded to FP32 exactly as the runtime upload rounds
them; a CPU test checks that the committed file still matches.  Degree 6 (784
entries per derivative matrix) keeps constant memory, and at degree 5 only the
kernels that the workloads use take the table (the kernel selects them), since
folding the tables into every unrolled node loop makes those translation units
take many minutes to compile.  Run as
``python -m paper_2012_13487_gb300.csrc.gen_ops_tables`` after a build.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "ops_tables.inc")
MAX_P = 5


def table(p):
    from paper_2012_13487_gb300 import fedbm as fb
    o = fb.fedbm_ref_operators(p)
    vals = np.concatenate([o["Dr"].ravel(), o["Ds"].ravel(), o["LIFT"].ravel()])
    return [float(np.float32(v)) for v in vals]


def render():
    lines = ["// Generated by gen_ops_tables.py from the library's operators: FP32 Dr, Ds",
             "// (row-major Np x Np) and LIFT (row-major Np x 3(p+1)) of the FEDBM_P of the",
             "// including translation unit, in the order of the runtime upload.  Do not edit."]
    for p in range(MAX_P + 1):
        lines.append("#%s FEDBM_P == %d" % ("if" if p == 0 else "elif", p))
        vals = table(p)
        lines.append("#define FEDBM_OPS32_TABLE \\")
        for i in range(0, len(vals), 4):
            chunk = ", ".join(v.hex() + "f" for v in vals[i:i + 4])
            lines.append("  %s%s \\" % (chunk, "," if i + 4 < len(vals) else ""))
        lines[-1] = lines[-1][:-2]
    lines.append("#endif")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write(render())
    print(OUT)
