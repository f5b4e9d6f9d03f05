"""The allocation-free solve entry point, checked against chol_solve.

chol_solve_noalloc serves callers that cannot allocate device memory (for example code that
must not call cudaMalloc while a stream is being captured into a CUDA graph, or that works
inside a device-memory budget owned by the host application). It keeps its workspace in a
fixed array of the library, so these tests call it through the C ABI twice in a row and
compare with the workspace-taking chol_solve on the same factor, within the tolerance of the
solve parity tests. The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

REL_X = 1e-12
BERR = 1e-14


def _fn():
    import paper_1402_6601_gb300 as chol
    f = ctypes.CDLL(chol.build.LIB).chol_solve_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p]
    return chol, f


@pytest.mark.parametrize("n,nrhs", [(1000, 70), (257, 1)])
def test_noalloc_solve_matches_solve_on_two_calls(n, nrhs):
    chol, f = _fn()
    A = synth.gram_spd(n, seed=31).numpy()
    B = synth.rhs(n, nrhs, seed=32).numpy()
    Ld = chol.colmajor(torch.from_numpy(A).to("cuda"))
    chol.factor(Ld, chol.opts(nb=128), check=True)
    Bd = chol.colmajor(torch.from_numpy(B).to("cuda"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        ref = Bd.clone()
        chol.solve(Ld, ref)
        got = Bd.clone()
        info = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        st = f(n, nrhs, Ld.data_ptr(), Ld.stride(1), got.data_ptr(), got.stride(1) if nrhs > 1 else n,
               info.data_ptr(), stream)
        assert st == 0, "call %d returned %d" % (call, st)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        X, Xref = got.cpu().numpy(), ref.cpu().numpy()
        assert oracle.rel_frobenius(X, Xref) <= REL_X
        assert oracle.backward_error(A, X, B) <= BERR


def test_noalloc_rejects_problems_beyond_its_array():
    chol, f = _fn()
    # ceil(n/32) * ceil(nrhs/32) above 32704 does not fit; rejected before any launch (the
    # pointers pass the argument checks and are never dereferenced)
    fake = ctypes.c_void_p(256)
    st = f(32705 * 32, 1, fake, 32705 * 32, fake, 32705 * 32, None, None)
    assert st == -5
    st = f(-1, 1, None, 1, None, 1, None, None)
    assert st == -1
