"""The C ABI library loads and exports every entry point declared in
include/*.h; host-side argument checks run without a GPU (no compute call)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pic_[a-z0-9_]+)\s*\(",
                                text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1008_1685_gb300 import build as b

    b.build()
    import paper_1008_1685_gb300 as picrr

    return picrr.library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"pic_create", "pic_load_foil", "pic_inject_laser", "pic_step_n", "pic_spectra",
            "pic_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    import paper_1008_1685_gb300.binding as bnd

    assert names == set(bnd.SYMBOLS) | (names - set(bnd.SYMBOLS))
    assert set(bnd.SYMBOLS) <= names


def test_invalid_config_rejected_on_host(lib):
    import paper_1008_1685_gb300 as picrr

    for bad in (dict(cfl=1.0), dict(cfl=0.0), dict(cells_per_lambda=-1.0), dict(sort_interval=97),
                dict(source_node=1), dict(lambda_um=0.0)):
        kw = dict(length_lambda=4, cells_per_lambda=50, cfl=0.95)
        kw.update(bad)
        with pytest.raises(picrr.PicError) as e:
            picrr.Sim(**kw)
        assert e.value.status == -1


def test_destroy_null_and_null_handle_calls(lib):
    assert lib.pic_destroy(None) == 0
    assert lib.pic_step_n(None, 1, None) == -1
    assert lib.pic_energy(None, None) == -1
    out = C.c_void_p()
    assert lib.pic_create(None, C.byref(out)) == -1 and not out.value
    assert b"NULL" in lib.pic_last_error(None)


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout: a small C
    program built with the host compiler prints every field's offset and each
    struct's size, compared with the binding's."""
    import ctypes
    import shutil
    import subprocess

    from paper_1008_1685_gb300 import binding as B

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pic_config": B.Config, "pic_run_desc": B.RunDesc, "pic_stats_t": B.Stats,
               "pic_server_stats_t": B.ServerStats, "pic_electron_case": B.ElectronCase}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "picrr.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            cname, field, value = line.split()
            got[(cname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
