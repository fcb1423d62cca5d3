"""Host-side checks of the C-ABI library that need no GPU: it loads, it
exports every function include/kmedoids.h declares, the workspace size is
sane, and argument validation returns a status (no launch happens)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kmedoids.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2008_05171_gb300 import build as b
    b.build()
    import paper_2008_05171_gb300.kmedoids as km
    return km.load()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(km\w*|kmedoids\w*)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "kmedoids_run" in names and len(names) >= 8
    for name in names:
        assert hasattr(lib, name), name
    import paper_2008_05171_gb300.kmedoids as km
    assert sorted(km.EXPORTS) == names


def test_workspace_size(lib):
    import paper_2008_05171_gb300.kmedoids as km
    a = km.workspace_size(1000, 10, km.KM_I32)
    b = km.workspace_size(20000, 100, km.KM_F32)
    assert 0 < a < b
    assert km.workspace_size(10, 11, km.KM_F32) == 0  # k > n
    assert km.workspace_size(0, 1, km.KM_F32) == 0
    assert km.workspace_size(10, 2, 7) == 0           # unknown dtype
    o = km.options(variant="fastpam2")
    assert km.workspace_size(20000, 100, km.KM_F32, o) > b
    o = km.options(trace=1000)
    assert km.workspace_size(20000, 100, km.KM_F32, o) > b


def test_invalid_arguments_return_status(lib):
    import paper_2008_05171_gb300.kmedoids as km
    o = km.options()
    res = km.km_result()
    P = ctypes.c_void_p
    buf = (ctypes.c_char * 4096)()
    fake = ctypes.addressof(buf) + (256 - ctypes.addressof(buf) % 256) % 256
    cases = [
        (None, 1, 100, 100, 10, 1),      # D NULL
        (fake, 5, 100, 100, 10, 1),      # dtype
        (fake, 1, 100, 100, 0, 1),       # k = 0
        (fake, 1, 100, 100, 101, 1),     # k > n
        (fake, 1, 100, 99, 10, 1),       # ld < n
        (fake, 1, 100, 102, 10, 1),      # ld not a multiple of 4
        (fake + 4, 1, 100, 100, 10, 1),  # misaligned D
        (fake, 1, 100, 100, 10, 2),      # workspace too small
    ]
    for D, dt, n, ld, k, want in cases:
        st = lib.kmedoids_run(P(D), dt, n, ld, k, P(fake), None,
                              ctypes.byref(o), ctypes.byref(res), P(fake), 64,
                              None)
        assert st == want, (D, dt, n, ld, k, st)
        assert lib.kmedoids_last_error()
    for bad in (km.options(variant=9), km.options(tune=-2), km.options(tune=17)):
        st = lib.kmedoids_run(P(fake), 1, 100, 100, 10, P(fake), None,
                              ctypes.byref(bad), ctypes.byref(res), P(fake), 1 << 30,
                              None)
        assert st == 1


def test_version(lib):
    import paper_2008_05171_gb300.kmedoids as km
    assert "sm_103a" in km.version()


def test_invalid_arguments_of_the_newer_entry_points(lib):
    """16-bit stride rule, the initialisations' and the batched form's host
    checks: each returns its status before any device work."""
    import paper_2008_05171_gb300.kmedoids as km
    P = ctypes.c_void_p
    buf = (ctypes.c_char * 4096)()
    fake = ctypes.addressof(buf) + (256 - ctypes.addressof(buf) % 256) % 256
    o = km.options()
    res = km.km_result()
    # KM_U16 needs ld % 8 == 0 (16-byte rows)
    st = lib.kmedoids_run(P(fake), km.KM_U16, 100, 100, 10, P(fake), None, ctypes.byref(o),
                          ctypes.byref(res), P(fake), 1 << 30, None)
    assert st == 1 and b"multiple of 8" in lib.kmedoids_last_error()
    # distance-weighted initialisation: u NULL
    assert lib.kmedoids_init_weighted(P(fake), 1, 100, 100, 5, None, P(fake), P(fake),
                                      1 << 30, None) == 1
    # LAB: subsample size out of range, NULL ranks
    assert lib.kmedoids_init_lab(P(fake), 1, 100, 100, 5, 0, P(fake), P(fake), None,
                                 P(fake), 1 << 30, None) == 1
    assert lib.kmedoids_init_lab(P(fake), 1, 100, 100, 5, 5000, P(fake), P(fake), None,
                                 P(fake), 1 << 30, None) == 7
    assert lib.kmedoids_init_lab(P(fake), 1, 100, 100, 5, 8, None, P(fake), None,
                                 P(fake), 1 << 30, None) == 1
    # batched form: only FastPAM1 and FasterPAM
    bad = km.options(variant="fastpam2")
    assert lib.kmedoids_run_batched(P(fake), P(fake), 1, P(fake), P(fake), ctypes.byref(bad),
                                    P(fake), 1 << 20, None) == 7
    # batched geometries: a table of five; tune outside it is rejected
    w, st = ctypes.c_int32(), ctypes.c_int32()
    assert lib.kmedoids_batched_geometry_info(1, ctypes.byref(w), ctypes.byref(st)) == 0
    assert (w.value, st.value) == (16, 4)
    assert lib.kmedoids_batched_geometry_info(6, None, None) == -1
    assert lib.kmedoids_batched_geometry_info(0, None, None) == -1
    bad_tune = km.options(tune=6)
    assert lib.kmedoids_run_batched(P(fake), P(fake), 1, P(fake), P(fake),
                                    ctypes.byref(bad_tune), P(fake), 1 << 20, None) == 1
    g = ctypes.c_int32()
    assert lib.kmedoids_batched_autotune(P(fake), P(fake), 1, P(fake), P(fake), None,
                                         P(fake), 16, None, ctypes.byref(g), None) == 2
    assert lib.kmedoids_batched_autotune(P(fake), P(fake), 1, P(fake), P(fake), None,
                                         P(fake), 1 << 20, None, None, None) == 1
    # batch + CLARA in one enqueue: host checks before any device work
    assert lib.kmedoids_batched_clara_workspace_size(0, 5, 4, 100) > 0
    assert lib.kmedoids_batched_clara_workspace_size(3, 5, 4, 100) >= \
        lib.kmedoids_batched_clara_workspace_size(0, 5, 4, 100)
    assert lib.kmedoids_batched_clara_workspace_size(0, 5, 4, 4) == 0
    cres = ctypes.c_void_p(fake)
    args = [None, None, 0, None, None, P(fake), 1000, 8, 5, 4, 100, P(fake), P(fake), None,
            None, cres, None, P(fake), 1 << 30, None]
    a = list(args)
    a[2] = -1
    assert lib.kmedoids_run_batched_clara(*a) == 1        # negative count
    a = list(args)
    a[8] = 200                                             # k > 128
    assert lib.kmedoids_run_batched_clara(*a) == 1
    a = list(args)
    a[15] = None                                           # no result record
    assert lib.kmedoids_run_batched_clara(*a) == 1
    a = list(args)
    a[18] = 1024                                           # workspace too small
    assert lib.kmedoids_run_batched_clara(*a) == 2
    # a negative wait limit is rejected by every form that waits
    neg = km.options(wait_limit_ns=-1)
    assert lib.kmedoids_run(P(fake), km.KM_F32, 100, 100, 10, P(fake), None, ctypes.byref(neg),
                            ctypes.byref(res), P(fake), 1 << 30, None) == 1
    assert b"wait_limit_ns" in lib.kmedoids_last_error()
    assert lib.kmedoids_run_features(P(fake), 1000, 32, 32, 10, P(fake), None,
                                     ctypes.byref(neg), ctypes.byref(res), P(fake), 1 << 30,
                                     None) == 1
    # wait self-test: kind, limit and workspace checked before any launch
    assert lib.kmedoids_wait_selftest(4, 1000, P(fake), 512, None) == 1
    assert lib.kmedoids_wait_selftest(-1, 1000, P(fake), 512, None) == 1
    assert lib.kmedoids_wait_selftest(0, -1, P(fake), 512, None) == 1
    assert lib.kmedoids_wait_selftest(0, 10 ** 11, P(fake), 512, None) == 1
    assert lib.kmedoids_wait_selftest(0, 1000, P(fake), 256, None) == 1
    assert lib.kmedoids_wait_selftest(0, 1000, P(fake + 8), 512, None) == 1
    assert lib.kmedoids_wait_selftest(0, 1000, None, 512, None) == 1
    # bichromatic form: sizes checked before any launch
    ws_bi = lib.kmedoids_bichromatic_workspace_size
    assert ws_bi(0, 10, 2, km.KM_F32, None) == 0
    assert ws_bi(10, 20, 11, km.KM_F32, None) == 0          # k > m
    assert ws_bi(10, 20, 3, 7, None) == 0                   # dtype
    assert ws_bi(10, 20, 3, km.KM_F32, None) > 0
    assert ws_bi(3000, 20, 3, km.KM_F32, None) > ws_bi(10, 20, 3, km.KM_F32, None)
    for m_, n_, k_, ld_ in ((0, 20, 2, 20), (10, 0, 2, 20), (10, 20, 11, 20), (10, 20, 2, 18)):
        assert lib.kmedoids_run_bichromatic(P(fake), km.KM_F32, m_, n_, ld_, k_, P(fake), None,
                                            None, ctypes.byref(res), P(fake), 1 << 30,
                                            None) == 1, (m_, n_, k_, ld_)
    # matrix upload: dtype, pointers and sizes checked before any CUDA call
    up = lib.kmedoids_upload_matrix
    assert up(P(fake), 100, 7, 100, P(fake), 100, None) == 1          # dtype
    assert up(None, 100, km.KM_F32, 100, P(fake), 100, None) == 1     # host NULL
    assert up(P(fake), 100, km.KM_F32, 100, None, 100, None) == 1     # D NULL
    assert up(P(fake), 100, km.KM_F32, 0, P(fake), 100, None) == 1    # n = 0
    assert up(P(fake), 99, km.KM_F32, 100, P(fake), 100, None) == 1   # host_ld < n
    assert up(P(fake), 100, km.KM_F32, 100, P(fake), 99, None) == 1   # ld < n
    assert up(P(fake), 1 << 40, km.KM_F32, 1 << 30, P(fake), 1 << 40, None) == 1
    assert b"too large" in lib.kmedoids_last_error()


def _c_struct_fields(name):
    """Field names of `typedef struct name { ... } name;` in the header, in
    declaration order (comments stripped; `int32_t a, b;` gives a and b)."""
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), txt, flags=re.S)
    assert body, name
    fields = []
    for decl in body.group(1).split(";"):
        decl = decl.strip()
        if decl:  # [const] type [*]name[, [*]name ...]
            rest = re.match(r"(?:const\s+)?\w+\s*(.*)", decl, flags=re.S).group(1)
            fields += [x.strip().lstrip("*").strip() for x in rest.split(",")]
    return fields


@pytest.mark.parametrize("struct", ["km_options", "km_result"])
def test_ctypes_structs_match_the_header(struct, tmp_path):
    """The binding's ctypes mirrors have the header's fields in the same
    order at the same offsets, and the same size, as a C compiler lays them
    out (gcc on this host)."""
    import shutil
    import subprocess
    import paper_2008_05171_gb300.kmedoids as km
    cls = getattr(km, struct)
    names = [f for f, _ in cls._fields_]
    assert names == _c_struct_fields(struct)
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"kmedoids.h\"\n"
                   "int main(void) {\n  printf(\"%%zu\\n\", sizeof(%s));\n" % struct +
                   "".join("  printf(\"%%zu\\n\", offsetof(%s, %s));\n" % (struct, f)
                           for f in names) + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, f).offset for f in names]


def test_bounds_checking_build_loads_and_exports_the_same_symbols(tmp_path):
    """The -DKM_BOUNDS_CHECK variant (libkmedoids_bounds.so) builds, exports
    every declared function, reports itself through kmedoids_bounds_checked
    and validates arguments as the regular build does; the binding loads it
    when KMEDOIDS_BOUNDS_CHECK=1."""
    import subprocess
    import sys
    from paper_2008_05171_gb300 import build as b
    path = b.build(bounds_check=True)
    assert path.endswith("libkmedoids_bounds.so")
    code = (
        "import ctypes, sys\n"
        "sys.path.insert(0, %r)\n"
        "import paper_2008_05171_gb300.kmedoids as km\n"
        "assert km.LIB_PATH.endswith('libkmedoids_bounds.so'), km.LIB_PATH\n"
        "lib = km.load()\n"
        "assert lib.kmedoids_bounds_checked() == 1\n"
        "for name in km.EXPORTS: getattr(lib, name)\n"
        "P = ctypes.c_void_p\n"
        "assert lib.kmedoids_wait_selftest(4, 1000, P(1 << 20), 512, None) == 1\n"
        "print('ok')\n" % ROOT)
    env = dict(os.environ, KMEDOIDS_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
    import paper_2008_05171_gb300.kmedoids as km
    if os.environ.get("KMEDOIDS_BOUNDS_CHECK") != "1":
        assert km.load().kmedoids_bounds_checked() == 0
