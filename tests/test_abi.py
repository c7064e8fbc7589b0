"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/pi.h declares (no compute call: no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pi_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1601_00159_gb300 import build as b
    import paper_1601_00159_gb300 as pkg
    path = b.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} is declared in pi.h but not exported"
    assert sorted(pkg.EXPORTED) == sorted(names)
    pkg.load_library(path)


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1601_00159_gb300 as pkg
    saved = pkg._lib
    pkg._lib = None
    try:
        try:
            pkg.load_library(str(tmp_path / "missing.so"))
        except RuntimeError as e:
            assert "not built" in str(e)
        else:
            raise AssertionError("loading a missing library must raise")
    finally:
        pkg._lib = saved


def test_result_struct_layout():
    # pi_result_t is 16 bytes: u64 value, u32 status, u32 reserved.
    src = open(os.path.join(ROOT, "include", "pi.h")).read()
    m = re.search(r"typedef struct \{(.*?)\} pi_result_t;", src, flags=re.S)
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    fields = [tuple(x.split()) for x in body.replace("\n", " ").split(";") if x.strip()]
    assert fields == [("uint64_t", "value"), ("uint32_t", "status"), ("uint32_t", "reserved")]


def test_info_struct_matches_binding():
    import paper_1601_00159_gb300 as pkg
    # 3 u64 + 4 u32 + 34 u64 + 8 u64
    assert ctypes.sizeof(pkg.PiInfo) == 3 * 8 + 4 * 4 + 34 * 8 + 8 * 8
    assert ctypes.sizeof(pkg.PiConfig) == 4 * 4 + 2 * 8 + 4 * 4


def _header_fields(name):
    """(type, field) pairs of `typedef struct {...} name;` in include/pi.h."""
    src = open(os.path.join(ROOT, "include", "pi.h")).read()
    m = re.search(r"typedef struct \{((?:[^{}])*?)\} " + name + ";", src, flags=re.S)
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    out = []
    for decl in body.split(";"):
        parts = decl.split()
        if not parts:
            continue
        field = re.sub(r"\[.*\]", "", parts[-1])
        out.append((" ".join(parts[:-1]), field))
    return out


def test_config_structs_match_binding():
    """The binding's ctypes structs name the header's fields in the header's order."""
    import paper_1601_00159_gb300 as pkg
    for cname, cls in (("pi_config_t", pkg.PiConfig), ("pi_multi_class_t", pkg.PiMultiClass),
                       ("pi_info_t", pkg.PiInfo)):
        hdr = [f for _, f in _header_fields(cname)]
        assert hdr == [f for f, _ in cls._fields_], cname
