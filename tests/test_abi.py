"""The C ABI without a GPU: libmp.so builds for sm_103a, loads, exports every
function include/mp.h declares, and its structs have the layout the Python
binding marshals."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2302_13590_gb300 import mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(mp_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("mp_field_load", "mp_release_group", "mp_track", "mp_get_endpoints", "mp_get_timeseries"):
        assert required in names


def test_every_declared_call_cites_its_passage():
    """Each call of the boundary names the passage of the paper it follows
    (or says that it is infrastructure with no passage) in a comment that
    ends directly above its declaration."""
    src = open(HEADER).read()
    for name in declared_functions():
        m = re.search(r"^(?:const\s+)?\w+\**\s+\**" + name + r"\s*\(", src, flags=re.M)
        assert m, name
        before = src[:m.start()].rstrip()
        assert before.endswith("*/"), f"{name}: no comment directly above its declaration"
        comment = before[before.rindex("/*"):]
        assert "Passage:" in comment, f"{name}: comment names no passage"
        body = comment.split("Passage:", 1)[1]
        assert re.search(r"(Introduction|Methods|Results|Conclusions|none)", body), name


def test_library_loads_and_exports_every_declared_symbol():
    lib = mp.load_library()
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in mp.SIGNATURES, f"binding lacks {n}"
    # the binding declares nothing the header does not
    assert set(mp.SIGNATURES) <= set(names)


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu\\n", sizeof(mp_field_desc), offsetof(mp_field_desc, origin),
         offsetof(mp_field_desc, qx), offsetof(mp_field_desc, flags), sizeof(mp_ts_record));
  printf("%zu %zu %zu %zu\\n", sizeof(mp_release_desc), offsetof(mp_release_desc, lo),
         offsetof(mp_release_desc, seed), offsetof(mp_release_desc, id_offset));
  printf("%zu %zu %zu %zu\\n", sizeof(mp_track_opts), offsetof(mp_track_opts, t_stop),
         offsetof(mp_track_opts, block), offsetof(mp_track_opts, flags));
  printf("%zu %zu %zu %zu\\n", sizeof(mp_endpoints), sizeof(mp_stats), offsetof(mp_stats, kernel_ms),
         offsetof(mp_stats, path_points));
  printf("%zu %zu %zu %zu\\n", offsetof(mp_track_opts, path_capacity), sizeof(mp_path_record),
         offsetof(mp_path_record, seq), offsetof(mp_track_opts, weak_sink_fraction));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(prog)])
    got = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().split("\n") if l]
    F, R, T = mp.FieldDesc, mp.ReleaseDesc, mp.TrackOpts
    assert got[0] == [ctypes.sizeof(F), F.origin.offset, F.qx.offset, F.flags.offset, mp.TS_RECORD.itemsize]
    assert got[1] == [ctypes.sizeof(R), R.lo.offset, R.seed.offset, R.id_offset.offset]
    assert got[2] == [ctypes.sizeof(T), T.t_stop.offset, T.block.offset, T.flags.offset]
    assert got[3] == [ctypes.sizeof(mp.Endpoints), ctypes.sizeof(mp.Stats), mp.Stats.kernel_ms.offset,
                      mp.Stats.path_points.offset]
    assert got[4] == [T.path_capacity.offset, mp.PATH_RECORD.itemsize, mp.PATH_RECORD.fields["seq"][1],
                      T.weak_sink_fraction.offset]


def test_no_device_calls_fail_cleanly_without_gpu():
    """Host-side argument checks answer before any device work."""
    lib = mp.load_library()
    out = ctypes.c_void_p()
    assert lib.mp_ctx_create(0, None) == -1
    assert lib.mp_field_load(None, None, ctypes.byref(out)) == -1
    assert b"NULL" in lib.mp_last_error()
    o = mp.make_opts(mode=mp.MODE_TIMESERIES, times=[1.0, 2.0])
    b = mp.mp_query_bytes(o, 1000)
    assert b >= 1000 * 2 * 32
