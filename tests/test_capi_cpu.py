"""Host-side checks of the C ABI library (no GPU needed): it loads and exports every
function that include/kifmm.h declares, and the Python binding marshals arguments only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "kifmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kifmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__  # noqa: F401
    from paper_1605_01715_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_declared_symbols():
    from paper_1605_01715_gb300 import capi
    assert sorted(capi.exported_symbols()) == declared()


def test_version_and_error_string(lib):
    lib.kifmm_version.restype = ctypes.c_char_p
    lib.kifmm_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.kifmm_version()
    assert isinstance(lib.kifmm_last_error(), bytes)


def test_null_arguments_rejected_without_a_gpu(lib):
    """Argument checks run on the host before any CUDA call."""
    out = ctypes.c_void_p()
    lib.kifmm_tree_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.kifmm_tree_build(None, 10, None, 0, 8, None, ctypes.byref(out)) == -1
    assert not out.value
    lib.kifmm_fmm_matvec.argtypes = [ctypes.c_void_p] * 4
    assert lib.kifmm_fmm_matvec(None, None, None, None) == -1
    lib.kifmm_tree_destroy.argtypes = [ctypes.c_void_p]
    assert lib.kifmm_tree_destroy(None) == 0
    lib.kifmm_fmm_matvec_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p]
    assert lib.kifmm_fmm_matvec_host(None, None, None, 1, None) == -1


def test_forest_arguments_rejected_without_a_gpu(lib):
    """kifmm_forest_build checks sizes and offsets on the host before any CUDA call."""
    import numpy as np
    out = ctypes.c_void_p()
    f = lib.kifmm_forest_build
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    fake = ctypes.c_void_p(0x1000)             # never dereferenced: the checks fail first
    for off, n in (([1, 10], 10), ([0, 5, 5, 10], 10), ([0, 4, 9], 10), ([0, 10], 11)):
        a = np.asarray(off, dtype=np.int64)
        assert f(fake, n, a.ctypes.data, len(off) - 1, 16, None, ctypes.byref(out)) == -1
        assert not out.value
    a = np.zeros(2, dtype=np.int64)
    assert f(fake, 10, a.ctypes.data, 0, 16, None, ctypes.byref(out)) == -1        # no instances
    assert f(None, 10, a.ctypes.data, 1, 16, None, ctypes.byref(out)) == -1        # NULL points


def _unit_surface(p):
    """The boundary points of the p x p x p grid on [-1, 1]^3, x outermost, then y, then z
    (the numbering include/kifmm.h states for kifmm_up_skeleton)."""
    import numpy as np
    g = np.linspace(-1.0, 1.0, p)
    return np.array([(x, y, z) for x in g for y in g for z in g
                     if min(abs(abs(x) - 1), abs(abs(y) - 1), abs(abs(z) - 1)) < 1e-12])


def _check_potentials(p, n, seed):
    """Potentials at the up-check surface (2.95 half-widths) of n unit monopoles and n
    unit dipoles at random points inside the box: two Q x n matrices, by numpy."""
    import numpy as np
    c = 2.95 * _unit_surface(p)
    rng = np.random.default_rng(seed)
    y = rng.uniform(-1.0, 1.0, (n, 3))
    nrm = rng.standard_normal((n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    d = c[:, None, :] - y[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    return 1.0 / r, (d * nrm[None]).sum(-1) / r ** 3


def test_up_skeleton_interpolates_source_potentials(lib):
    """The S2U skeleton (kifmm_up_skeleton, an interpolative decomposition the mixed
    form uses in place of the paper's full check surface) reproduces, from its k
    points, the potential of sources inside the box at every one of the Q check points:
    exactly at k = Q, to about 1e-9 (monopoles) and 1e-7 (dipoles) of the largest value
    at the k = 384 that p = 10 plans use, and less well with fewer points."""
    import numpy as np
    from paper_1605_01715_gb300 import kifmm_up_skeleton
    p = 10
    Q = 6 * (p - 1) ** 2 + 2
    mono, dip = _check_potentials(p, 1500, seed=11)
    errs = {}
    for k in (300, 384, Q):
        idx, E, kt = kifmm_up_skeleton(p, k)
        assert idx.shape == (k,) and E.shape == (Q, k)
        assert len(set(idx.tolist())) == k and idx.min() >= 0 and idx.max() < Q
        assert np.array_equal(E[idx], np.eye(k))          # skeleton rows interpolate themselves
        assert 0 < kt <= Q
        errs[k] = [float((np.abs(A - E @ A[idx]).max(0) / np.abs(A).max(0)).max()) for A in (mono, dip)]
    assert errs[Q][0] < 1e-12 and errs[Q][1] < 1e-12
    assert errs[384][0] < 2e-8 and errs[384][1] < 5e-7
    assert errs[300][0] > errs[384][0] and errs[300][1] > errs[384][1]


def test_up_skeleton_sizes_and_arguments(lib):
    """Pivot counts above 1e-9: every point at low order (p = 6: Q = 152), fewer than Q
    from p = 8 on.  Out-of-range p or k are rejected on the host."""
    from paper_1605_01715_gb300 import KifmmError, kifmm_up_skeleton
    kts = {p: kifmm_up_skeleton(p, 1)[2] for p in (6, 8, 10, 11)}
    assert kts[6] == 152
    for p in (8, 10, 11):
        assert kts[p] < 6 * (p - 1) ** 2 + 2
    assert kts[8] < kts[10] < kts[11]
    for p, k in ((1, 1), (17, 1), (10, 0), (10, 489)):
        with pytest.raises(KifmmError):
            kifmm_up_skeleton(p, k)


def test_stats_structs_match_the_header(tmp_path):
    """The binding's ctypes mirrors of kifmm_tree_stats and kifmm_plan_stats have the C
    header's size and field offsets (compiled with the host C compiler)."""
    import shutil
    import subprocess
    from paper_1605_01715_gb300.capi import PlanStats, TreeStats
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    structs = (("kifmm_tree_stats", TreeStats), ("kifmm_plan_stats", PlanStats))
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "kifmm.h"', "int main(void) {"]
    for cname, cls in structs:
        body.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            body.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    body += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(body) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for cname, cls in structs:
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)
