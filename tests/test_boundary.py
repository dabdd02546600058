"""The C-ABI library builds, loads on a machine without a GPU and exports
every entry point declared in include/isc.h; the binding fails loudly when
the library is missing (no CPU fallback)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "isc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1811_11992_gb300 import build, isc
    lib_path = build.build()
    lib = isc.load_library(lib_path)
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(isc._SIGS), set(names) ^ set(isc._SIGS)


def test_status_strings_without_gpu():
    from paper_1811_11992_gb300 import isc
    lib = isc.load_library()
    assert lib.isc_status_string(0) == b"ok"
    assert lib.isc_status_string(-4) == b"singular diagonal block"
    o = isc.default_options()
    assert o.restart == 30 and o.prec == 2 and o.decouple == 1


def test_missing_library_fails_loudly(tmp_path):
    from paper_1811_11992_gb300 import isc
    saved = isc._lib
    isc._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            isc.load_library(str(tmp_path / "nope.so"))
    finally:
        isc._lib = saved


def test_ctypes_structures_match_the_header(tmp_path):
    """Every structure the binding declares has the header's size and field
    offsets (a C probe compiled against include/isc.h)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1811_11992_gb300 import isc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(isc, n) for n in dir(isc)
               if n.startswith("isc_") and isinstance(getattr(isc, n), type)
               and issubclass(getattr(isc, n), ctypes.Structure)]
    assert len(structs) >= 10
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "isc.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'printf("{S.__name__} size %zu\\n", sizeof({S.__name__}));')
        for f in S._fields_:
            lines.append(f'printf("{S.__name__} {f[0]} %zu\\n", offsetof({S.__name__}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for S in structs:
        assert got[(S.__name__, "size")] == ctypes.sizeof(S), S.__name__
        for f in S._fields_:
            assert got[(S.__name__, f[0])] == getattr(S, f[0]).offset, (S.__name__, f[0])


@pytest.mark.parametrize("lang", ["c99", "c++17"])
def test_header_compiles_cleanly(tmp_path, lang):
    """include/isc.h is a self-contained C99 header (and valid C++): no warnings
    with -Wall -Wextra -pedantic, and a C caller can pass the handle returned by
    isc_create to every other call (one struct isc_handle type throughout)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c99" else "g++")
    if cc is None:
        pytest.skip("no compiler")
    src = tmp_path / ("use.c" if lang == "c99" else "use.cpp")
    src.write_text('#include "isc.h"\n'
                   "int use(const isc_grid* g, const isc_rock* r, const isc_fluid* f, const isc_reactions* x,\n"
                   "        const isc_wells* w) {\n"
                   "  isc_options o; struct isc_handle* h = 0; isc_newton_info info;\n"
                   "  isc_default_options(&o);\n"
                   "  if (isc_create(g, r, f, x, w, &o, &h) != ISC_OK) return 1;\n"
                   "  int st = isc_newton_step(h, 1.0, &info);\n"
                   "  isc_destroy(h);\n"
                   "  return st;\n"
                   "}\n")
    std = "-std=c99" if lang == "c99" else "-std=c++17"
    subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                    str(src), "-o", str(tmp_path / "use.o")], check=True)


def _prototypes():
    """name -> (return type text, [parameter texts]) for every prototype in the header."""
    src = open(os.path.join(ROOT, "include", "isc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(isc_[a-z0-9_]+)\s*\(([^;{)]*)\)\s*;", src):
        params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(2)] = (m.group(1).strip(), params)
    return out


def test_binding_signatures_match_the_prototypes():
    """The ctypes declarations of the binding have the header's parameter count,
    pointer-ness of every parameter and return kind (void / int / pointer)."""
    import ctypes as C
    from paper_1811_11992_gb300 import isc
    protos = _prototypes()
    assert set(protos) == set(isc._SIGS)
    for name, (res, args) in isc._SIGS.items():
        ret, params = protos[name]
        assert len(args) == len(params), (name, params)
        for a, p in zip(args, params):
            is_ptr = "*" in p or "[" in p  # an array parameter is a pointer
            ct_ptr = a is C.c_void_p or a is C.c_char_p or (isinstance(a, type) and issubclass(a, C._Pointer))
            assert is_ptr == ct_ptr, (name, p, a)
            if not is_ptr:  # scalars: the same width and kind
                base = p.replace("const", "").split()[0]
                want = {"int32_t": C.c_int32, "int": C.c_int, "double": C.c_double, "int64_t": C.c_int64,
                        "size_t": C.c_size_t}[base]
                assert C.sizeof(a) == C.sizeof(want) and (a is C.c_double) == (want is C.c_double), (name, p, a)
        if ret.endswith("void") and "*" not in ret:
            assert res is None, name
        elif "*" in ret:
            assert res in (C.c_char_p, C.c_void_p), name
        else:
            assert res in (C.c_int, C.c_int32, C.c_int64), (name, ret)


def _enum_values():
    src = open(os.path.join(ROOT, "include", "isc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(ISC_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_binding_constants_match_the_header_enums():
    """The binding's and the input generator's constants equal the header's enum values."""
    import isc_inputs as inp
    from paper_1811_11992_gb300 import isc
    e = _enum_values()
    assert isc.KRYLOV == {"gmres": e["ISC_KRYLOV_GMRES"], "bicgstab": e["ISC_KRYLOV_BICGSTAB"]}
    assert isc.PREC["none"] == e["ISC_PREC_NONE"] and isc.PREC["bjacobi"] == e["ISC_PREC_BJACOBI"]
    assert isc.PREC["bilu0"] == e["ISC_PREC_BILU0"] and isc.PREC["cpr"] == e["ISC_PREC_CPR"]
    assert isc.PRECISION == {"fp64": e["ISC_PRECISION_FP64"], "mixed": e["ISC_PRECISION_MIXED"],
                             "mixed_fgmres": e["ISC_PRECISION_MIXED_FGMRES"]}
    assert isc.ORTH == {"cgs2": e["ISC_ORTH_CGS2"], "cgs1": e["ISC_ORTH_CGS1"]}
    defines = dict(re.findall(r"#define\s+(ISC_[A-Z0-9_]+)\s+(\d+)", open(os.path.join(ROOT, "include", "isc.h")).read()))
    assert isc.NOALLOC_MAX_CELLS == int(defines["ISC_NOALLOC_MAX_CELLS"])
    statuses = {v for k, v in e.items() if k == "ISC_OK" or k.startswith("ISC_ERR_")}
    assert set(isc.STATUS) == statuses
    assert len(isc.K_CLASSES) == e["ISC_K_COUNT"]
    for i, name in enumerate(isc.K_CLASSES):
        assert e["ISC_K_" + name.upper()] == i, name
    assert (inp.RXN_OIL_OXIDATION, inp.RXN_CRACKING, inp.RXN_COKE_OXIDATION) == (
        e["ISC_RXN_OIL_OXIDATION"], e["ISC_RXN_CRACKING"], e["ISC_RXN_COKE_OXIDATION"])
    assert (inp.WELL_RATE_INJECTOR, inp.WELL_BHP_PRODUCER, inp.WELL_COUPLED_PRODUCER, inp.WELL_COUPLED_INJECTOR) == (
        e["ISC_WELL_RATE_INJECTOR"], e["ISC_WELL_BHP_PRODUCER"], e["ISC_WELL_COUPLED_PRODUCER"],
        e["ISC_WELL_COUPLED_INJECTOR"])
    assert (inp.CTRL_BHP, inp.CTRL_WATER_RATE, inp.CTRL_OIL_RATE, inp.CTRL_LIQUID_RATE, inp.CTRL_GAS_RATE,
            inp.CTRL_TOTAL_RATE) == tuple(e["ISC_CTRL_" + k] for k in ("BHP", "WATER_RATE", "OIL_RATE",
                                                                       "LIQUID_RATE", "GAS_RATE", "TOTAL_RATE"))


def test_every_handle_call_rejects_a_null_handle_without_a_gpu():
    """Every entry point that takes the handle answers a NULL one before any
    CUDA work: ISC_ERR_INVALID_ARG from the int-returning calls, nothing from
    isc_destroy, 0 from the size and count queries and a message from
    isc_last_error."""
    import ctypes as C
    from paper_1811_11992_gb300 import isc
    lib = isc.load_library()
    protos = _prototypes()
    seen = 0
    for name, (ret, params) in protos.items():
        if not params or "isc_handle" not in params[0] or "**" in params[0]:
            continue
        fn = getattr(lib, name)
        args = [None]
        for p in params[1:]:
            if "*" in p or "[" in p:
                args.append(None)
            elif "double" in p:
                args.append(1.0)
            else:
                args.append(1)
        res = fn(*args)
        if name == "isc_destroy":
            assert res is None
        elif name == "isc_last_error":
            assert res and b"null" in res
        elif name in ("isc_num_cells", "isc_nnzb", "isc_num_coupled_wells"):
            assert res == 0, name
        else:
            assert res == _enum_values()["ISC_ERR_INVALID_ARG"], name
        seen += 1
    assert seen >= 40
