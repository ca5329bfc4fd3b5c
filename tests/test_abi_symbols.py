"""The C-ABI library loads without a GPU and exports every symbol include/krp.h declares."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "krp.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(krp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2507_23207_gb300 as K
    from paper_2507_23207_gb300 import build

    build.build()
    return K.load_library()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["krp_gen_factors", "krp_sketch_mode", "krp_tucker_rhosvd",
                 "krp_tucker_sthosvd", "krp_block_hankel_lowrank"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2507_23207_gb300 as K
    assert sorted(K.EXPORTED) == declared_symbols()


def test_abi_version_and_status_strings(lib):
    import paper_2507_23207_gb300 as K
    assert K.krp_abi_version() == 2
    assert lib.krp_status_string(K.KRP_EINVAL) == b"KRP_EINVAL"
    assert lib.krp_status_string(K.KRP_ETIMEOUT) == b"KRP_ETIMEOUT"


def test_null_context_is_rejected_without_a_gpu(lib):
    import paper_2507_23207_gb300 as K
    assert lib.krp_destroy(None) == K.KRP_EINVAL
    assert lib.krp_set_stream(None, None) == K.KRP_EINVAL
    assert lib.krp_last_error(None) == b"null context"


def test_without_a_gpu_the_library_fails_loudly(lib):
    """No CPU fallback: with no usable GPU, creating a context is an error
    (KRP_ECUDA from the C ABI, KrpError from the binding), so no entry point
    that needs a context can run."""
    import ctypes as C
    import torch
    import paper_2507_23207_gb300 as K
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.krp_create(C.byref(h), 0, None) == K.KRP_ECUDA
    assert not h.value
    with pytest.raises(K.KrpError) as e:
        K.Context(0, 0)
    assert e.value.status == K.KRP_ECUDA


def test_noalloc_qr_checks_its_arguments_before_touching_the_device(lib):
    """krp_qr_noalloc rejects sizes beyond its fixed scratch (and l outside
    1..64, m < l, null pointers) before any CUDA call, so the rejection is
    the same with or without a GPU."""
    import ctypes as C
    import paper_2507_23207_gb300 as K
    p = C.c_void_p(256)  # never dereferenced: every call below is rejected first
    assert lib.krp_qr_noalloc(p, 16384, 48, p, None, None) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(p, 100, 65, p, None, None) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(p, 3, 4, p, None, None) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(p, 100, 0, p, None, None) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(None, 8, 4, p, None, None) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(p, 8, 4, None, None, None) == K.KRP_EINVAL
