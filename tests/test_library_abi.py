"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/asss.h declares (no compute calls here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "asss.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(asss_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("asss_setup", "asss_solve", "asss_solve_adjoint", "asss_destroy", "asss_mrs",
              "asss_skew_symmetrizer", "asss_skew_lanczos"):
        assert f in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_06954_gb300 as pkg
    L = pkg.lib()
    missing = [f for f in _declared() if not hasattr(L, f)]
    assert not missing, missing
    assert set(pkg.EXPORTED) <= set(_declared())


def test_options_defaults_round_trip():
    import paper_2009_06954_gb300.binding as b
    o = b.default_options()
    assert o.k_lanczos == 20 and o.gamma == 1.0 and o.outer_tol == 1e-8 and o.restart == 60
    assert o.precision == b.ASSS_PREC_FP64 and o.outer == b.ASSS_OUTER_TFQMR


def test_status_strings():
    import paper_2009_06954_gb300 as pkg
    L = pkg.lib()
    assert L.asss_status_str(0) == b"ok"
    assert L.asss_status_str(8) == b"device wait timed out"


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of asss_csr, asss_options and asss_stats have the C sizes and
    field offsets (compiled from include/asss.h with the host C compiler)."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2009_06954_gb300 import binding as B
    structs = {"asss_csr": B.CSR, "asss_options": B.Options, "asss_stats": B.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "asss.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_batched_packing_follows_the_abi_layout():
    """System m occupies [off_m * nrhs, (off_m + n_m) * nrhs) of the concatenated vector,
    column-major n_m x nrhs inside (the layout asss_solve_batched documents)."""
    import numpy as np
    from paper_2009_06954_gb300.binding import BatchSolver
    bs = object.__new__(BatchSolver)  # the packing needs only the sizes
    bs.sizes = [3, 5, 2]
    bs.offsets = np.concatenate([[0], np.cumsum(bs.sizes)]).astype(np.int64)
    bs.total = int(bs.offsets[-1])
    nrhs = 4
    rng = np.random.default_rng(0)
    blocks = [rng.standard_normal((n, nrhs)) for n in bs.sizes]
    v = bs.pack(blocks)
    assert v.shape == (bs.total * nrhs,)
    for m, (o, n) in enumerate(zip(bs.offsets[:-1], bs.sizes)):
        for c in range(nrhs):
            np.testing.assert_array_equal(v[o * nrhs + c * n: o * nrhs + (c + 1) * n], blocks[m][:, c])
    for a, b in zip(bs.unpack(v, nrhs), blocks):
        np.testing.assert_array_equal(a, b)


def test_output_buffers_are_checked_on_the_host():
    """solve_adjoint's caller-owned outputs: float64, contiguous, the right length
    (checked before any call into the library)."""
    import numpy as np
    import torch
    from paper_2009_06954_gb300.binding import _check_out
    _check_out("lam", np.empty(10), 10)
    _check_out("dA", torch.empty(7, dtype=torch.float64), 7)
    for bad in (np.empty(9), np.empty(10, dtype=np.float32), np.empty((10, 2))[:, 0],
                torch.empty(10, dtype=torch.float32), torch.empty(20, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            _check_out("lam", bad, 10)
