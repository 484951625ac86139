"""The C ABI library loads without a GPU and exports every declared call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(pdlp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_04756_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_call():
    from paper_2106_04756_gb300 import _abi
    assert set(_declared()) == set(_abi._SIGNATURES)


def _param_counts():
    out = {}
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for name, params in re.findall(r"\b(pdlp_\w+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
                p = params.strip()
                out[name] = 0 if p in ("", "void") else p.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    from paper_2106_04756_gb300 import _abi
    counts = _param_counts()
    for name, (args, _) in _abi._SIGNATURES.items():
        assert len(args) == counts[name], (name, len(args), counts[name])


def test_default_options_are_the_papers(lib):
    import paper_2106_04756_gb300 as P
    o = P.default_options()
    assert (o.beta_suff, o.beta_nec, o.beta_art) == (0.9, 0.1, 0.5)
    assert o.pw_smoothing == 0.5 and o.eval_every == 40 and o.ruiz_iters == 10
    assert o.pock_chambolle == 1 and o.rel_tol == 1e-8 and o.primal_importance == 1.0


def test_create_rejects_bad_arguments_before_any_device_work(lib):
    import paper_2106_04756_gb300 as P
    from paper_2106_04756_gb300 import _abi
    out = C.c_void_p()
    rc = _abi.load().pdlp_create(None, None, None, None, None, None, None, C.byref(out))
    assert rc == _abi.PDLP_ERR_INVALID_ARG and not out.value
    # negative sizes
    rp = np.zeros(2, np.int32)
    csr = _abi.pdlp_csr(-1, 3, 0, rp.ctypes.data, None, None)
    z = np.zeros(3)
    rc = _abi.load().pdlp_create(C.byref(csr), z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                                 np.zeros(3, np.uint8).ctypes.data, None, C.byref(out))
    assert rc == _abi.PDLP_ERR_INVALID_ARG
    assert b"CSR" in _abi.load().pdlp_last_error(None)
    # a bad option
    o = P.default_options(precision=7)
    csr = _abi.pdlp_csr(1, 1, 0, rp.ctypes.data, None, None)
    rc = _abi.load().pdlp_create(C.byref(csr), z.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data,
                                 np.zeros(3, np.uint8).ctypes.data, C.byref(o), C.byref(out))
    assert rc == _abi.PDLP_ERR_INVALID_ARG


def test_binding_struct_layout_matches_the_header(tmp_path):
    """Field offsets and sizes of pdlp_options / pdlp_result / pdlp_csr as the
    C compiler lays them out from include/pdlp.h, against the ctypes mirrors."""
    import shutil
    import subprocess
    from paper_2106_04756_gb300 import _abi
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"pdlp_options": _abi.pdlp_options, "pdlp_result": _abi.pdlp_result, "pdlp_csr": _abi.pdlp_csr}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdlp.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'  printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = {}
    for line in got:
        if line:
            s, f, v = line.split()
            want[(s, f)] = int(v)
    for sname, cls in structs.items():
        assert C.sizeof(cls) == want[(sname, "size")], sname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == want[(sname, fname)], (sname, fname)


def test_no_cpu_fallback_without_a_gpu(lib):
    """Without a CUDA device every compute entry point raises PdlpError
    (PDLP_ERR_CUDA) instead of returning a result computed some other way."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import lpgen
    import paper_2106_04756_gb300 as P
    lp = lpgen.small_planted()
    calls = [lambda: P.solve(lp), lambda: P.solve(lp, precision=P.PDLP_FP32_REFINE),
             lambda: P.solve(lp, presolve=1), lambda: P.Context.from_lp(lp, unroll_T=5),
             lambda: P.solve_batch([lp, lpgen.small_planted()])]
    for call in calls:
        with pytest.raises(P.PdlpError) as e:
            call()
        assert e.value.code == P.PDLP_ERR_CUDA, e.value


def test_binding_checks_array_lengths_before_the_library_reads_them(lib):
    """The C ABI takes bare pointers; the binding rejects an input of the
    wrong length (which the library would read past) and an output of the
    wrong length or dtype (which it would write past) with ValueError."""
    import copy
    import torch
    import lpgen
    import paper_2106_04756_gb300 as P
    base = lpgen.small_planted()
    for field, cut in (("row_ptr", 1), ("col_idx", 1), ("c", 1), ("q", 1), ("l", 1), ("u", 1), ("ineq", 1)):
        lp = copy.deepcopy(base)
        setattr(lp, field, getattr(lp, field)[:-cut])
        with pytest.raises(ValueError):
            P.Context.from_lp(lp)
    lp = copy.deepcopy(base)
    lp.c = torch.as_tensor(lp.c[:-1])
    with pytest.raises(ValueError):
        P.Context.from_lp(lp)
    with pytest.raises(ValueError):
        P._out(torch.zeros(base.n, dtype=torch.float32), base.n)
    with pytest.raises(ValueError):
        P._out(np.zeros(base.n - 1), base.n)
    assert P._in(np.zeros(4), np.float64, 4)[1].size == 4
