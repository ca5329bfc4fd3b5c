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
    assert header_layout["KRP_ABI_VERSION"] == 1
