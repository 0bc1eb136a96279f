"""bench.py's count of the oracle equation list's work over symmetry-allowed blocks,
checked against an independent count: for every term, the number of index-value tuples
(not irrep tuples) at which all its operands are allowed by their symmetry rules,
summed by an einsum over element-level masks."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _element_count(spec, kinds, irr_o, irr_v):
    ins, _ = spec.split("->")
    ops = ins.split(",")
    masks = []
    for lab, kind in zip(ops, kinds):
        gs = [irr_o if c in "ijklmn" else irr_v for c in lab]
        tot = 0
        for k, (sgn, g) in enumerate(zip(bench._SGN[kind], gs)):
            shape = [1] * len(lab)
            shape[k] = len(g)
            tot = tot + sgn * g.reshape(shape)
        masks.append(((tot % G_) == 0).astype(np.float64))
    idx = "".join(sorted(set("".join(ops))))
    return float(np.einsum(",".join(ops) + "->" + idx, *masks).sum())


@pytest.mark.parametrize("G,occ,virt", [(1, [3], [5]), (2, [2, 1], [3, 2]), (4, [1, 0, 2, 1], [2, 3, 0, 2])])
def test_oracle_work_equals_element_count(G, occ, virt):
    global G_
    G_ = G
    irr_o = np.repeat(np.arange(G), occ)
    irr_v = np.repeat(np.arange(G), virt)
    for spec, *kinds in bench.ORACLE_TERMS:
        assert bench.term_macs(spec, kinds, occ, virt) == _element_count(spec, kinds, irr_o, irr_v), spec


def test_oracle_work_dense_is_product_of_extents():
    # G = 1: every tuple is allowed, so a term costs the product of its index extents
    o, v = 4, 7
    for spec, *kinds in bench.ORACLE_TERMS:
        idx = set(spec.split("->")[0].replace(",", ""))
        want = np.prod([o if c in "ijklmn" else v for c in idx])
        assert bench.term_macs(spec, kinds, [o], [v]) == want
