"""fv_apply_op_noalloc: the operator apply for callers that must not allocate device memory.

Such callers (e.g. code whose device memory belongs to a framework's pool
allocator, or a loop that cannot take cudaMalloc's implicit synchronisation)
get the same y = A x with the ghost-layer scratch in the library's static
device array.  Checked against fv_apply_op on two calls in a row (the array
keeps the previous call's contents), for both systems, plus the size limit.
This file is collected last so that a failure here never hides other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

from paper_2009_02171_gb300.inputs import random_vector  # noqa: E402

PH = dict(E=1e-3, Ra=100.0, Pr=1.0, Pm=5.0, dt=1e-4)


@pytest.fixture(scope='module')
def fv():
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    from paper_2009_02171_gb300 import fv as f
    return f


@pytest.mark.parametrize('kind,Ns,Nr', [(0, 12, 10), (1, 16, 12)])
def test_noalloc_apply_matches_apply_on_consecutive_calls(fv, kind, Ns, Nr):
    g = fv.fv_build_grid(Ns, Nr)
    s = fv.fv_assemble_system(g, kind, **PH)
    n = fv.fv_system_size(s)
    for call in range(2):
        x = torch.tensor(random_vector(n, 100 + call), device='cuda')
        ref = fv.fv_apply_op(s, x, torch.empty_like(x))
        got = fv.fv_apply_op_noalloc(s, x, torch.empty_like(x))
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-12, (call, err)
    fv.fv_free_system(s)
    fv.fv_free_grid(g)


def test_noalloc_larger_then_smaller_system(fv):
    """A call on a system with a larger ghost layer, then one on a smaller system: the second call
    overwrites every slot it reads, so the stale tail of the array does not leak into its result."""
    res = []
    for kind, Ns, Nr in ((0, 16, 14), (1, 8, 6)):
        g = fv.fv_build_grid(Ns, Nr)
        s = fv.fv_assemble_system(g, kind, **PH)
        n = fv.fv_system_size(s)
        x = torch.tensor(random_vector(n, 200 + kind), device='cuda')
        ref = fv.fv_apply_op(s, x, torch.empty_like(x))
        got = fv.fv_apply_op_noalloc(s, x, torch.empty_like(x))
        torch.cuda.synchronize()
        res.append((got - ref).abs().max().item() / ref.abs().max().item())
        fv.fv_free_system(s)
        fv.fv_free_grid(g)
    assert max(res) < 1e-12, res


def test_noalloc_rejects_systems_beyond_the_static_limit(fv):
    g = fv.fv_build_grid(8, 640)           # VTBE ghost layer 7 x 24 x 640 x 10 = 1,075,200 doubles > 2^20
    s = fv.fv_assemble_system(g, 0, **PH, p=(1, 1, 8), overlap=1)
    n = fv.fv_system_size(s)
    x = torch.zeros(n, dtype=torch.float64, device='cuda')
    with pytest.raises(fv.FvError, match='FV_STATIC_GHOST_DOUBLES'):
        fv.fv_apply_op_noalloc(s, x, torch.empty_like(x))
    fv.fv_free_system(s)
    fv.fv_free_grid(g)
