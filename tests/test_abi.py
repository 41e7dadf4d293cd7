"""CPU-side checks of the C ABI: the library builds, loads, exports every
entry point the header declares, and rejects bad arguments on the host
without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(sdl_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_03800_gb300 import _build, sdl
    if not os.path.exists(sdl.LIB_PATH):
        _build.build()
    return sdl.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sdl_sparse_code", "sdl_update_D1", "sdl_update_D2", "sdl_iterate",
                 "sdl_create", "sdl_destroy", "sdl_status"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in sdl.h but not exported"


def test_binding_covers_every_declared_symbol():
    from paper_2007_03800_gb300 import sdl
    for name in declared_functions():
        assert name in sdl.SIGNATURES or name in ("sdl_strerror", "sdl_kernel_name"), name


def test_shape_support_rules(lib):
    assert lib.sdl_shape_supported(8, 8, 16, 16, 4) == 1
    assert lib.sdl_shape_supported(12, 12, 24, 24, 6) == 1
    assert lib.sdl_shape_supported(16, 64, 32, 128, 10) == 1
    assert lib.sdl_shape_supported(16, 16, 32, 32, 8) == 1
    assert lib.sdl_shape_supported(8, 8, 16, 16, 33) == 0      # s above the register Cholesky
    assert lib.sdl_shape_supported(2, 2, 16, 16, 5) == 0       # s > p1*p2
    assert lib.sdl_shape_supported(8, 8, 256, 16, 4) == 0      # no tile shape
    assert lib.sdl_shape_supported(65, 8, 16, 16, 4) == 0


def test_tiling_listing_and_pinning_arguments(lib):
    from paper_2007_03800_gb300 import sdl
    t12 = sdl.tilings(12, 12, 24, 24, 6)
    assert len(t12) >= 3 and len(set(t12)) == len(t12)
    assert len(sdl.tilings(8, 8, 16, 16, 4)) >= 2 and len(sdl.tilings(16, 16, 32, 32, 8)) >= 2
    assert sdl.tilings(10, 10, 20, 20, 5) == []               # generic kernel only
    assert not set(t12) & set(sdl.tilings(8, 8, 16, 16, 4))
    assert lib.sdl_tilings(12, 12, 24, 24, 6, None, -1) == -1
    assert lib.sdl_set_tiling(None, 12, 12, 24, 24, 6, t12[0], 0) == -1
    assert lib.sdl_tune_tiling(None, None, 12, 12, 10, None, 24, None, 24, 6, None, None) == -1
    assert lib.sdl_tune_log(None, None, None, None, 0) == -1


def test_host_argument_errors_without_gpu(lib):
    from paper_2007_03800_gb300 import sdl
    assert lib.sdl_sparse_code(None, None, 8, 8, 10, None, 16, None, 16, 4, 0.0,
                               None, None, None, None, None) == -1
    assert lib.sdl_iterate(None, None, 8, 8, 10, None, 16, None, 16, 4, 0.0,
                           None, None, None, None, None) == -1
    assert lib.sdl_ortho_iterate(None, None, 8, 8, 10, None, None, 4, 0.0, None, None, None,
                                 None, None) == -1
    assert lib.sdl_ortho_sparse_code(None, None, 8, 8, 10, None, None, 4, 0.0, None, None, None,
                                     None, None) == -1
    assert lib.sdl_gemm_bf16(None, None, 64, None, 64, 128, 128, 64, 1.0, None, 0, None, 0, 0,
                             None, 0, None, 0, None, 0, None) == -1
    assert lib.sdl_gemm_bf16_terms(None, None, 64, None, 64, 2, 128, 128, 64, 1.0, None, 0, None,
                                   0, 0, None, 0, None, 0, None, 0, None) == -1
    assert lib.sdl_create(None, 0) == -1
    assert lib.sdl_destroy(None) == 0
    assert lib.sdl_strerror(-4) == b"normal matrix not positive definite"
    assert sdl.ERRORS[-7] == "SDL_ERR_UNSUPPORTED"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.sdl_create(ctypes.byref(h), 0) == -2
    assert h.value is None


def test_binding_constants_match_the_header():
    """Error codes, batch flags and precision flags of the binding are the
    values the header defines (parsed from the header text)."""
    from paper_2007_03800_gb300 import sdl
    text = open(HEADER).read()
    errs = dict((int(v), k) for k, v in re.findall(r"^\s*(SDL_ERR_\w+)\s*=\s*(-?\d+)", text, flags=re.M))
    assert errs == sdl.ERRORS
    defs = dict((k, int(v)) for k, v in re.findall(r"^#define\s+(SDL_\w+)\s+(\d+)", text, flags=re.M))
    assert sdl.NUM_KERNEL_KINDS == defs["SDL_NUM_KERNEL_KINDS"]
    for name in ("BATCH_AUTOTUNE", "BATCH_GRAPH", "BATCH_RETUNE"):
        assert getattr(sdl, name) == defs["SDL_" + name], name
    ctx_cls = sdl.Context
    for name in ("PREC_FP32", "PREC_BF16_CORR", "PREC_NO_RESCORE", "PREC_FP64_SOLVE"):
        assert getattr(ctx_cls, name) == defs["SDL_" + name], name


def test_summed_gemm_binding_checks_operands_on_the_host():
    """gemm_bf16_terms rejects operand lists of unequal length, empty lists,
    non-BF16 operands and pairs of differing shapes before any library call."""
    import torch

    from paper_2007_03800_gb300 import sdl
    a = torch.zeros((128, 64), dtype=torch.bfloat16)
    b = torch.zeros((96, 64), dtype=torch.bfloat16)
    for A, B in (([a, a], [b]), ([], []), ([a.float()], [b]), ([a, a[:, :32]], [b, b]),
                 ([a, a], [b, b[:64]])):
        with pytest.raises(ValueError):
            sdl.gemm_bf16_terms(None, A, B)
