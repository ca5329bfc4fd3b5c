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
    assert K.krp_abi_version() == 1
    assert lib.krp_status_string(K.KRP_EINVAL) == b"KRP_EINVAL"
    assert lib.krp_status_string(K.KRP_ETIMEOUT) == b"KRP_ETIMEOUT"


def test_null_context_is_rejected_without_a_gpu(lib):
    import paper_2507_23207_gb300 as K
    assert lib.krp_destroy(None) == K.KRP_EINVAL
    assert lib.krp_set_stream(None, None) == K.KRP_EINVAL
    assert lib.krp_last_error(None) == b"null context"
