"""Host-side helpers that change an instance's layout or list coordinate blocks
(no step of the method): checked on the CPU."""
import numpy as np
import pytest
import torch

from paper_2002_00352_gb300 import gen
from paper_2002_00352_gb300.categorical import expand_categorical, fold_decisions
from paper_2002_00352_gb300.solver import cyclic_blocks


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_categorical_expansion_layout(layout):
    """Every copy of item j carries item j's profit and consumption (dense and CSR
    layouts give the same expanded instance), and each local set holds the copies
    of its items."""
    inst = gen.random_small(40, 4, 3, seed=5, device="cpu", layout=layout, frac=0.3)
    inst.S, inst.C = [0b0011, 0b1100, 0b1111], [1, 2, 3]
    u = [2, 1, 3, 1]
    big = expand_categorical(inst, u)
    p, b = inst.to_dense_numpy()
    p2, b2 = big.to_dense_numpy()
    src = np.repeat(np.arange(4), u)
    assert big.M == sum(u)
    assert np.array_equal(p2, p[:, src]) and np.array_equal(b2, b[:, src, :])
    assert big.S == [0b000111, 0b111000 | 0b1000000, 0b1111111]
    assert big.C == inst.C


def test_categorical_expansion_rejects_bad_bounds():
    inst = gen.random_small(5, 3, 2, seed=1, device="cpu", layout="dense")
    for u in ([1, 2], [1, 0, 2], [30, 30, 5]):
        with pytest.raises(ValueError):
            expand_categorical(inst, u)


def test_fold_decisions_counts_copies():
    x2 = torch.tensor([[1, 1, 0, 1, 0, 0], [0, 0, 1, 1, 1, 1]])
    assert fold_decisions(x2, [2, 1, 3]).tolist() == [[2, 0, 1], [0, 1, 3]]


def test_cyclic_blocks_order():
    assert cyclic_blocks(3, 2) == [[0], [1], [2], [0], [1], [2]]
    assert cyclic_blocks(1, 0) == []
