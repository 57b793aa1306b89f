"""Host-side checks of the C ABI (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    hdr = ""
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            hdr += open(os.path.join(inc, f)).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def libqp():
    import paper_1512_07437_b300.build as b
    b.build()
    import paper_1512_07437_b300 as qp
    return qp.lib()


def test_library_exports_every_declared_entry_point(libqp):
    names = _declared_symbols()
    assert "qp_posteriors" in names and "qp_server_poll" in names
    for n in names:
        assert hasattr(libqp, n), n
    out = subprocess.run(["nm", "-D", "--defined-only",
                          os.path.join(ROOT, "paper_1512_07437_b300", "libqp.so")],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qp_[a-z0-9_]+)", out))
    assert set(names) <= exported


def test_build_targets_sm_103a_only():
    import paper_1512_07437_b300.build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layout_matches_header(libqp, tmp_path):
    """ctypes mirrors must match the C structs: every field offset and every
    struct size as the C compiler lays out include/qp.h."""
    import shutil
    import subprocess
    import paper_1512_07437_b300.qp as q
    structs = [q.qp_family, q.qp_params, q.qp_result, q.qp_server_stats]
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qp.h"', 'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in st._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.splitlines())
    for st in structs:
        name = st.__name__
        assert int(out[name]) == ctypes.sizeof(st), name
        for fname, _ in st._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(st, fname).offset, f"{name}.{fname}"


def test_no_device_fails_loudly(libqp):
    """Without a usable GPU the product path raises; it never computes on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import synth
    import paper_1512_07437_b300 as qp
    fam = synth.star_family(1, 3, (20, 30), 0.3)
    with pytest.raises(qp.QpError):
        qp.qp_posteriors(fam.residues, fam.offsets, synth.default_params())


def test_invalid_inputs_rejected_on_host(libqp):
    """Malformed families and parameters are rejected before any device work."""
    import synth
    import paper_1512_07437_b300 as qp
    prm = synth.default_params()
    fam = synth.star_family(1, 3, (20, 30), 0.3)
    bad_offsets = fam.offsets.copy()
    bad_offsets[2] = bad_offsets[1]            # empty sequence
    with pytest.raises(qp.QpError) as e:
        qp.qp_posteriors(fam.residues, bad_offsets, prm)
    assert e.value.code == 1
    with pytest.raises(qp.QpError) as e:      # k < 2
        qp.qp_posteriors(fam.residues[:10], np.array([0, 10]), prm)
    assert e.value.code == 1
    for field, value in (("threshold", 0.0), ("threshold", 1.5), ("temperature", -1.0)):
        bad = prm.replace(**{field: value})
        with pytest.raises(qp.QpError) as e:
            qp.qp_posteriors(fam.residues, fam.offsets, bad)
        assert e.value.code == 1, field
    long_res = np.full((1 << 20) + 11, ord("A"), dtype=np.uint8)     # one sequence over 2^20
    with pytest.raises(qp.QpError) as e:
        qp.qp_posteriors(long_res, np.array([0, 10, long_res.size]), prm)
    assert e.value.code == 1
    bad = prm.replace(pi=np.array([0.5, 0.1, 0.1, 0.1, 0.1]))
    with pytest.raises(qp.QpError) as e:
        qp.qp_posteriors(fam.residues, fam.offsets, bad)
    assert e.value.code == 1


def test_guide_tree_rejects_bad_input_on_host(libqp):
    """qp_guide_tree checks k and its pointers before touching a device, and
    without a device it fails rather than computing on the CPU."""
    import paper_1512_07437_b300 as qp
    with pytest.raises(qp.QpError) as e:
        qp.qp_guide_tree(np.zeros((1, 1)))
    assert e.value.code == 1
    L = qp.lib()
    m = np.zeros(4, dtype=np.int32)
    h = np.zeros(2)
    assert L.qp_guide_tree(None, 3, 0, 0, None, m.ctypes.data, h.ctypes.data) == 1
    assert L.qp_guide_tree(np.zeros(9).ctypes.data, 46341, 0, 0, None, m.ctypes.data, h.ctypes.data) == 1
    with pytest.raises(ValueError):
        qp.qp_guide_tree(np.zeros((2, 3)))
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(qp.QpError):
            qp.qp_guide_tree(np.ones((3, 3)))


def test_server_without_device_fails_loudly(libqp):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import synth
    import paper_1512_07437_b300 as qp
    with pytest.raises(qp.QpError):
        qp.Server(synth.default_params(), 1 << 30)


def test_static_limit_matches_header():
    """The Python binding's copy of QP_STATIC_MAX_LEN must be the header's."""
    hdr = open(os.path.join(ROOT, "include", "qp.h")).read()
    m = re.search(r"#define\s+QP_STATIC_MAX_LEN\s+(\d+)", hdr)
    assert m, "QP_STATIC_MAX_LEN is not defined in qp.h"
    from paper_1512_07437_b300 import qp as binding
    assert binding.QP_STATIC_MAX_LEN == int(m.group(1))
