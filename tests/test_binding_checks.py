"""The Python binding refuses output buffers the C entry points would overrun.

The C calls write into caller-owned output buffers (host or device) whose size
they cannot see; the binding checks dtype, layout, writability and size first.
CPU only: every case below is refused before the library is called, so the
handle is a stand-in that owns no device state.
"""
import numpy as np
import pytest

import paper_2212_04259_gb300 as F
from paper_2212_04259_gb300.fbn import _need_out

N_VARS = 5


def _handle(n=N_VARS, arity=3):
    return F.Handle(None, n, 10, np.full(n, arity, dtype=np.uint8))


@pytest.mark.parametrize("bad", [
    np.zeros((N_VARS - 1, N_VARS), dtype=np.uint8),                  # too small
    np.zeros((N_VARS, N_VARS), dtype=np.int32),                      # wrong dtype
    np.zeros((N_VARS, 2 * N_VARS), dtype=np.uint8)[:, ::2],           # not contiguous
])
def test_skeleton_adj_out_refused(bad):
    with pytest.raises(ValueError, match="adj_out"):
        F.fbn_learn_skeleton(_handle(), 0.05, -1, adj_out=bad)


def test_read_only_adj_out_refused():
    a = np.zeros((N_VARS, N_VARS), dtype=np.uint8)
    a.setflags(write=False)
    with pytest.raises(ValueError, match="adj_out"):
        F.fbn_learn_skeleton(_handle(), 0.05, -1, adj_out=a)


def test_torch_adj_out_checked():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="adj_out"):
        F.fbn_learn_skeleton(_handle(), 0.05, -1, adj_out=torch.zeros((N_VARS, N_VARS), dtype=torch.int64))
    with pytest.raises(ValueError, match="adj_out"):
        F.fbn_learn_skeleton(_handle(), 0.05, -1, adj_out=torch.zeros((N_VARS, N_VARS - 1), dtype=torch.uint8))
    with pytest.raises(ValueError, match="adj_out"):
        F.fbn_learn_skeleton(_handle(), 0.05, -1,
                             adj_out=torch.zeros((N_VARS, N_VARS), dtype=torch.uint8).t()[:, :-1])


def test_batch_adj_out_count_and_sizes():
    hs = [_handle(4), _handle(6)]
    with pytest.raises(ValueError, match="one buffer per handle"):
        F.fbn_learn_skeleton_batch(hs, 0.05, -1, adj_out=[np.zeros((4, 4), dtype=np.uint8)])
    with pytest.raises(ValueError, match=r"adj_out\[1\]"):
        F.fbn_learn_skeleton_batch(hs, 0.05, -1, adj_out=[np.zeros((4, 4), dtype=np.uint8),
                                                          np.zeros((5, 5), dtype=np.uint8)])


def test_sharded_adj_out_refused():
    with pytest.raises(ValueError, match="adj_out"):
        F.fbn_learn_skeleton_sharded(_handle(), 0.05, -1, own=None, exchange=None,
                                     adj_out=np.zeros(3, dtype=np.uint8))


def test_pairwise_counts_out_refused():
    h = _handle(arity=3)   # M = 15 one-hot rows: the Gram needs 225 int32
    with pytest.raises(ValueError, match="out"):
        F.fbn_pairwise_counts(h, out=np.zeros((15, 14), dtype=np.int32))
    with pytest.raises(ValueError, match="out"):
        F.fbn_pairwise_counts(h, out=np.zeros((15, 15), dtype=np.uint8))


def test_accepted_buffers():
    _need_out(np.zeros((3, 3), dtype=np.uint8), "a", np.uint8, 9)
    _need_out(np.zeros(20, dtype=np.int32), "a", np.int32, 9)   # larger is fine
    torch = pytest.importorskip("torch")
    _need_out(torch.zeros((3, 3), dtype=torch.uint8), "a", np.uint8, 9)
    _need_out(torch.zeros(9, dtype=torch.int32), "a", np.int32, 9)
