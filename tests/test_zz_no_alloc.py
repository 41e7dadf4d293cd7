"""sdl_sparse_code_static: the allocation-free sparse coder.

It serves callers that must not allocate device memory once running (their
GPU memory comes from a pre-sized pool they own, or cudaMalloc's implicit
synchronisation is unacceptable in their loop).  Its output must equal the
context-based sdl_sparse_code on the same inputs, call after call, since the
static scratch array it shares across calls is rewritten each time.
This file is collected last so that a stopping run has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2007_03800_gb300 import sdl, synth
from parity import COEF_RTOL, to_gpu_problem

pytestmark = pytest.mark.gpu


def _problem(seed, p, n, s, N):
    Y, _, _, _, _ = synth.kron_model(N, p, p, n, n, s, 20.0, seed=seed)
    D1, D2 = synth.init_dictionaries(p, p, n, n, seed=seed + 1)
    return to_gpu_problem(Y, D1, D2)


def test_static_matches_context_entry_point_two_calls(gpu_ctx):
    # two calls in a row with different shapes and data: the second must not
    # see anything the first left in the shared scratch
    for seed, p, n, s, N in ((3, 12, 24, 6, 5000), (4, 8, 16, 4, 3001)):
        Yg, D1g, D2g = _problem(seed, p, n, s, N)
        ref = gpu_ctx.sparse_code(Yg, D1g, D2g, s)
        assert gpu_ctx.status() == 0
        got = sdl.sparse_code_static(Yg, D1g, D2g, s)
        torch.cuda.synchronize()
        assert torch.equal(got.support, ref.support)
        assert torch.equal(got.nnz, ref.nnz)
        c_ref = ref.coef.cpu().numpy().astype(np.float64)
        c_got = got.coef.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(c_got - c_ref, axis=1) / np.maximum(np.linalg.norm(c_ref, axis=1), 1e-30)
        assert rel.max() < COEF_RTOL
        e_ref, e_got = ref.res_energy.cpu().numpy(), got.res_energy.cpu().numpy()
        assert np.allclose(e_got, e_ref, rtol=1e-5, atol=1e-6)
        assert sdl.static_status() == 0


def test_static_generic_path_and_no_energy_output(gpu_ctx):
    """A signal array that is not 16-byte aligned (a view one float in) runs
    the generic coder instead of the bulk-copy one, and res_energy may be
    omitted: both still equal the context-based coder."""
    Yg, D1g, D2g = _problem(5, 12, 24, 6, 2001)
    flat = torch.empty(Yg.numel() + 1, dtype=torch.float32, device="cuda:0")
    Yv = flat[1:].view(Yg.shape[0], Yg.shape[2], Yg.shape[1]).transpose(1, 2)   # column-major signals
    Yv.copy_(Yg)
    assert Yv.data_ptr() % 16 != 0
    ref = gpu_ctx.sparse_code(Yg, D1g, D2g, 6)
    out = sdl.Codes.empty(Yg.shape[0], 6, "cuda:0", with_energy=False)
    got = sdl.sparse_code_static(Yv, D1g, D2g, 6, out=out)
    torch.cuda.synchronize()
    assert torch.equal(got.support, ref.support) and torch.equal(got.nnz, ref.nnz)
    rel = (np.linalg.norm(got.coef.cpu().numpy() - ref.coef.cpu().numpy(), axis=1) /
           np.maximum(np.linalg.norm(ref.coef.cpu().numpy(), axis=1), 1e-30))
    assert rel.max() < COEF_RTOL
    assert sdl.static_status() == 0


def test_static_records_nonfinite_signals(gpu_ctx):
    """A NaN signal gets nnz = 0 and is reported by sdl_static_status, once."""
    Yg, D1g, D2g = _problem(6, 8, 16, 4, 300)
    Yg[17, 2, 3] = float("nan")
    got = sdl.sparse_code_static(Yg, D1g, D2g, 4)
    assert sdl.ERRORS[sdl.static_status()] == "SDL_ERR_NONFINITE"
    assert sdl.static_status() == 0
    nnz = got.nnz.cpu().numpy()
    assert nnz[17] == 0 and np.all(np.delete(nnz, 17) == 4)


def test_static_rejects_sizes_beyond_its_scratch(gpu_ctx):
    Yg, D1g, D2g = to_gpu_problem(np.zeros((4, 16, 64)), *synth.init_dictionaries(16, 64, 32, 128))
    with pytest.raises(sdl.SDLError) as e:
        sdl.sparse_code_static(Yg, D1g, D2g, 10)        # 32^2 + 128^2 > 8192 floats
    assert e.value.code == -8
    assert sdl.lib().sdl_strerror(-8) == b"problem exceeds the static scratch capacity"
