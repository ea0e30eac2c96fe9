"""The C ABI library loads, exports every function include/cdmt.h declares, and
rejects bad arguments with a status (no GPU needed: validation happens before
any CUDA call)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for h in os.listdir(HEADER_DIR):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(cdmt_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def cdmt():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1607_00909_gb300 as m
    return m


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("cdmt_plan", "cdmt_plan_ex", "cdmt_plan_info", "cdmt_execute", "cdmt_execute_host",
              "cdmt_destroy", "cdmt_strerror", "cdmt_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(cdmt):
    out = subprocess.run(["nm", "-D", "--defined-only", cdmt.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared() - exported
    assert not missing, missing
    for n in _declared():
        assert hasattr(cdmt.lib(), n)


def test_binding_names_match_header(cdmt):
    for n in _declared():
        assert callable(getattr(cdmt, n)), n


def test_status_strings(cdmt):
    assert cdmt.cdmt_strerror(0) == "success"
    assert cdmt.cdmt_strerror(cdmt.CDMT_EINVAL) == "invalid argument"
    assert cdmt.cdmt_strerror(12345) == "unknown status"


@pytest.mark.parametrize("kw,msg", [
    (dict(nsub=0), "nsub"),
    (dict(nchan=12), "nchan"),
    (dict(nchan=64), "nchan"),
    (dict(nint=0), "nint"),
    (dict(dm_list=[]), "ndm"),
    (dict(bw_sub=-1.0), "bw_sub"),
    (dict(f_centre=0.01), "lowest frequency"),
    (dict(dm_list=[0.0, float("nan")]), "finite"),
])
def test_plan_rejects_bad_arguments(cdmt, kw, msg):
    args = dict(nsub=1, nsamp=1 << 17, f_centre=135.0, bw_sub=0.1953125, dm_list=[0.0, 5.0], nchan=8, nint=4)
    args.update(kw)
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.cdmt_plan(args["nsub"], args["nsamp"], args["f_centre"], args["bw_sub"], args["dm_list"],
                       args["nchan"], args["nint"])
    assert e.value.status == cdmt.CDMT_EINVAL
    assert msg in str(e.value)
    assert msg in cdmt.cdmt_last_error(None)


def test_plan_rejects_unsupported_precision(cdmt):
    o = cdmt.cdmt_opts()
    o.precision = 77
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.cdmt_plan_ex(1, 1 << 17, 135.0, 0.1953125, [0.0], 8, 4, o)
    assert e.value.status == cdmt.CDMT_ENOTSUP


def test_null_handles(cdmt):
    lib = cdmt.lib()
    assert lib.cdmt_plan_info(None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_execute(None, None, None, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_execute_host(None, None, None, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_destroy(None) == cdmt.CDMT_OK
    assert lib.cdmt_plan_ex(None, 1, 1, 1.0, 1.0, None, 0, 8, 1, None) == cdmt.CDMT_EINVAL


def test_null_handles_of_the_8bit_and_incoherent_entry_points(cdmt):
    lib = cdmt.lib()
    assert lib.cdmt_redigitise(None, None, None, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_redigitise_sk(None, None, None, None, 3.0, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_execute_host_u8(None, None, None, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_incoherent(None, None, 0.0, 0.0, 1, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_plan_group(None, 0, None, None, None, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_inject_timeout(None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_server_save_beam(None, 0, None, None) == cdmt.CDMT_EINVAL
    assert lib.cdmt_server_restore_beam(None, 0, None, 0) == cdmt.CDMT_EINVAL


@pytest.mark.parametrize("limit_ms", [0.0, -1.0, 1001.0, float("nan")])
def test_selftest_wait_rejects_limits_outside_range(cdmt, limit_ms):
    # checked before any device call: the wait must stay short
    import ctypes
    g, w = ctypes.c_int(), ctypes.c_double()
    assert cdmt.lib().cdmt_selftest_wait(limit_ms, 0, ctypes.byref(g), ctypes.byref(w)) == cdmt.CDMT_EINVAL
    assert cdmt.lib().cdmt_selftest_wait(1.0, 0, None, None) == cdmt.CDMT_EINVAL


@pytest.mark.parametrize("groups", [-1, 3])
def test_plan_rejects_dm_groups_outside_the_list(cdmt, groups):
    # a group needs at least one DM trial; checked before any device call
    o = cdmt.cdmt_opts()
    o.dm_groups = groups
    with pytest.raises(cdmt.CdmtError) as e:
        cdmt.cdmt_plan_ex(1, 1 << 17, 135.0, 0.1953125, [0.0, 5.0], 8, 4, o)
    assert e.value.status == cdmt.CDMT_EINVAL
    assert "dm_groups" in str(e.value)


def test_struct_layouts_match_the_header(cdmt, tmp_path):
    """Every ctypes mirror of a header struct has the size and field offsets that
    the C compiler gives include/cdmt.h."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = [cdmt.cdmt_opts, cdmt.cdmt_info, cdmt.cdmt_beam, cdmt.cdmt_batch_opts, cdmt.cdmt_batch_tune,
               cdmt.cdmt_batch_beam_info, cdmt.cdmt_stream_desc, cdmt.cdmt_block_result, cdmt.cdmt_server_opts,
               cdmt.cdmt_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cdmt.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        n, f, v = line.split()
        got[(n, f)] = int(v)
    for st in structs:
        n = st.__name__
        assert got[(n, "size")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)


def test_binding_constants_match_header(cdmt):
    # the numeric #defines and enumerators the binding mirrors, read from the header text
    text = open(os.path.join(HEADER_DIR, "cdmt.h")).read()
    m = re.search(r"#define\s+CDMT_STATIC_SCRATCH_BYTES\s+\((\d+)u\s*\*\s*(\d+)u\s*\*\s*(\d+)u\)", text)
    assert m, "CDMT_STATIC_SCRATCH_BYTES not found"
    assert cdmt.CDMT_STATIC_SCRATCH_BYTES == int(m.group(1)) * int(m.group(2)) * int(m.group(3))
