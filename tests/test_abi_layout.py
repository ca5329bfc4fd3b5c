"""The ctypes binding agrees with include/krp.h byte for byte.

A small C program, compiled by the host C compiler against the header alone,
prints the size and field offsets of every struct the boundary passes by
pointer, and the value of every enum constant and flag macro.  The binding's
ctypes structures and constants must match them: a field added, dropped or
reordered on one side only would otherwise shift every later field of a
struct the library reads or writes.
"""

import ctypes as C
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "krp_phase_times": ("PhaseTimes", ["rng_ms", "sketch_ms", "qr_ms", "core_ms",
                                       "truncate_ms", "residual_ms", "total_ms"]),
    "krp_tucker_out": ("TuckerOut", ["core", "factors", "d", "core_dims", "rel_residual",
                                     "x_norm", "core_norm", "times"]),
    "krp_tucker_item": ("TuckerItem", ["X", "dims", "ranks", "seed", "core", "factors",
                                       "rel_residual"]),
    "krp_hankel_item": ("HankelItem", ["blocks", "m", "n", "s", "r", "ell_r", "ell_l",
                                       "seed", "U", "S", "V"]),
}

CONSTANTS = ["KRP_OK", "KRP_EINVAL", "KRP_ENOMEM", "KRP_ECUDA", "KRP_EUNSUPPORTED",
             "KRP_ETIMEOUT", "KRP_ENUMERIC", "KRP_F32", "KRP_BF16", "KRP_FP8_E4M3",
             "KRP_F64", "KRP_BF16X2", "KRP_MEMO", "KRP_TRUNCATE", "KRP_RESIDUAL",
             "KRP_TIMINGS", "KRP_MAXD", "KRP_DRAW_MEMO", "KRP_DRAW_FRESH_BASE",
             "KRP_DRAW_STHOSVD_BASE", "KRP_TAG_OMEGA", "KRP_TAG_PSI",
             "KRP_QR_NOALLOC_MAX_DOUBLES", "KRP_ABI_VERSION"]


def _probe_source():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "krp.h"',
             "int main(void) {", '  printf("{");']
    first = True
    for cname, (_, fields) in STRUCTS.items():
        for key, expr in [(f"{cname}.size", f"sizeof({cname})")] + [
                (f"{cname}.{f}", f"offsetof({cname}, {f})") for f in fields]:
            sep = "" if first else ","
            first = False
            lines.append(f'  printf("{sep}\\"{key}\\": %lld", (long long)({expr}));')
    for k in CONSTANTS:
        lines.append(f'  printf(",\\"{k}\\": %lld", (long long)({k}));')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    return "\n".join(lines)


@pytest.fixture(scope="module")
def header_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    src = d / "probe.c"
    exe = d / "probe"
    src.write_text(_probe_source())
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_the_header(header_layout, cname):
    import paper_2507_23207_gb300.krp as KB
    pyname, fields = STRUCTS[cname]
    cls = getattr(KB, pyname)
    assert [f[0] for f in cls._fields_] == fields, "field order differs from the header"
    assert C.sizeof(cls) == header_layout[f"{cname}.size"]
    for f in fields:
        assert getattr(cls, f).offset == header_layout[f"{cname}.{f}"], f


def test_constants_match_the_header(header_layout):
    import paper_2507_23207_gb300 as K
    for k in CONSTANTS:
        if k == "KRP_ABI_VERSION":
            continue
        assert getattr(K, k) == header_layout[k], k
    assert header_layout["KRP_ABI_VERSION"] == 2


# ---------------------------------------------------------------- prototypes --

_SCALARS = {"int": C.c_int, "unsigned": C.c_uint, "int64_t": C.c_int64,
            "uint64_t": C.c_uint64, "uint32_t": C.c_uint32, "size_t": C.c_size_t,
            "krp_dtype": C.c_int, "krp_status": C.c_int, "double": C.c_double}
_POINTEES = {"int": C.c_int, "int64_t": C.c_int64, "uint32_t": C.c_uint32,
             "double": C.c_double, "float": C.c_float, "char": C.c_char}


def _prototypes():
    import re
    with open(os.path.join(ROOT, "include", "krp.h")) as f:
        src = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    out = {}
    for ret, name, args in re.findall(
            r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(krp_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src):
        params = [a.strip() for a in args.split(",")]
        if params == ["void"]:
            params = []
        # drop the parameter name, keep the type
        types = [re.sub(r"\s*\b[A-Za-z_][A-Za-z0-9_]*$", "", p).strip() for p in params]
        out[name] = (ret.strip(), types)
    return out


def _check(ctype_str, ct, where):
    s = ctype_str.replace("const", " ").split()
    stars = "".join(s).count("*")
    base = "".join(s).replace("*", "")
    if base == "krp_ctx":               # an opaque pointer typedef
        stars += 1
        base = "void"
    if stars == 0:
        assert ct is _SCALARS[base], (where, ctype_str, ct)
        return
    if ct in (C.c_void_p, C.c_char_p):  # any data pointer passed as an address
        assert stars == 1, (where, ctype_str, ct)
        return
    pointee = ct._type_                 # POINTER(T)
    if stars >= 2:
        assert pointee is C.c_void_p, (where, ctype_str, ct)
    elif base in _POINTEES:
        assert C.sizeof(pointee) == C.sizeof(_POINTEES[base]), (where, ctype_str, ct)
    else:                               # a struct of the boundary: its own ctypes class
        assert base in STRUCTS and pointee.__name__ == STRUCTS[base][0], (where, ctype_str, ct)


def test_binding_signatures_match_the_header_prototypes():
    """Every argtypes/restype of the binding against the header's prototype:
    same arity, the same integer width for each scalar, and pointers where
    the header has pointers.  A 32-bit int passed for an int64_t (or an
    argument missing) would otherwise be accepted by ctypes silently."""
    import paper_2507_23207_gb300 as K
    from paper_2507_23207_gb300 import build
    build.build()                       # incremental: a no-op when up to date
    lib = K.load_library()
    protos = _prototypes()
    assert sorted(protos) == sorted(K.EXPORTED)
    for name, (ret, types) in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None and len(fn.argtypes) == len(types), name
        for i, (t, ct) in enumerate(zip(types, fn.argtypes)):
            _check(t, ct, f"{name} argument {i}")
        if ret == "const char*":
            assert fn.restype is C.c_char_p, name
        else:
            _check(ret, fn.restype, f"{name} result")
