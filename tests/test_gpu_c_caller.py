"""The C ABI used from C alone: a C99 program (generated here from the
combustion tube's inputs, every double written with 17 significant digits)
creates the handle, starts from the initial state, runs the time loop
(isc_run) and prints the final state; the result is the Python binding's
run of the same case through the same library, to the last bit."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import isc_inputs as inp


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_struct(var, obj, lens):
    """C assignments that rebuild a populated ctypes structure field by field;
    pointer fields become static arrays of the lengths in lens."""
    decl, body = [], []

    def value(v, t):
        if t in (C.c_double,):
            return repr(float(v))
        return str(int(v))

    def walk(expr, v, t):
        if isinstance(t, type) and issubclass(t, C.Array):
            for i in range(t._length_):
                walk(f"{expr}[{i}]", v[i], t._type_)
        else:
            body.append(f"  {expr} = {value(v, t)};")

    for name, t in obj._fields_:
        v = getattr(obj, name)
        if isinstance(t, type) and issubclass(t, C._Pointer):
            if not v:
                body.append(f"  {var}.{name} = 0;")
                continue
            n = lens[name]
            ct = "double" if t._type_ is C.c_double else "int32_t"
            arr = f"{var.replace('.', '_').replace('[', '_').replace(']', '')}_{name}"
            items = ", ".join(value(v[k], t._type_) for k in range(n))
            decl.append(f"static const {ct} {arr}[{n}] = {{{items}}};")
            body.append(f"  {var}.{name} = ({ct}*){arr};")
        elif t is C.c_void_p:
            body.append(f"  {var}.{name} = 0;")
        else:
            walk(f"{var}.{name}", v, t)
    return decl, body


T_END, DT0, DT_MAX = 600.0, 5.0, 150.0


def _program(tmp_path):
    """Generate and compile the C99 program; (executable, case)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1811_11992_gb300 import build, isc
    build.build()
    case = inp.tube_case()
    n = case.n
    keep = []
    g, rock, fl, rx, wells = isc.create_args(case, keep)
    decl, body = [], []
    for var, obj, lens in (("g", g, {"depth": n}), ("rock", rock, {"phi_ref": n, "perm": 3 * n}),
                           ("fl", fl, {}), ("rx", rx, {})):
        d, b = _c_struct(var, obj, lens)
        decl += d
        body += b
    for i, w in enumerate(case.wells):
        d, b = _c_struct(f"wl[{i}]", wells.wells[i], {"cells": len(w.cells), "WI": len(w.cells)})
        decl += d
        body += b
    ini = case.init
    ign = np.asarray(case.ignited, np.int32)
    t_end, dt0, dt_max = T_END, DT0, DT_MAX
    src = ["#include <stdio.h>", "#include <string.h>", '#include "isc.h"', ""] + decl + [
        "int main(void) {",
        "  isc_grid g; isc_rock rock; isc_fluid fl; isc_reactions rx; isc_wells wells;",
        f"  static isc_well wl[{len(case.wells)}];",
        "  memset(&g, 0, sizeof g); memset(&rock, 0, sizeof rock); memset(&fl, 0, sizeof fl);",
        "  memset(&rx, 0, sizeof rx); memset(wl, 0, sizeof wl);"] + body + [
        f"  wells.nw = {len(case.wells)}; wells.wells = wl;",
        "  isc_options o; isc_default_options(&o);",
        "  o.tol_newton = 1e-6; o.maxit_newton = 25; o.tol_lin = 1e-12; o.maxit_lin = 400;",
        "  struct isc_handle* h = 0;",
        "  int st = isc_create(&g, &rock, &fl, &rx, &wells, &o, &h);",
        '  if (st != ISC_OK) { printf("create %d %s\\n", st, isc_status_string(st)); return 1; }',
        f"  const double y_rest[3] = {{{', '.join(repr(float(v)) for v in ini['y_rest'])}}};",
        f"  static const int32_t ign[{max(1, len(ign))}] = {{{', '.join(str(int(v)) for v in ign) or '0'}}};",
        f"  st = isc_init_equilibrium(h, {ini['p']!r}, {ini['T']!r}, {ini['Sw']!r}, {ini['So']!r}, "
        f"{ini['x_LO']!r}, y_rest, {len(ign)}, ign, {ini['T_ignite']!r});",
        '  if (st != ISC_OK) { printf("init %d %s\\n", st, isc_last_error(h)); return 1; }',
        "  static double hist[1000]; isc_run_info info;",
        f"  st = isc_run(h, {t_end!r}, {dt0!r}, {dt_max!r}, 20.0, 0.2, 8, 1000, hist, &info);",
        '  if (st != ISC_OK) { printf("run %d %s\\n", st, isc_last_error(h)); return 1; }',
        f"  static double u[{8 * n}], coke[{n}];",
        "  if (isc_get_state(h, u, coke) != ISC_OK) return 1;",
        '  printf("%d %d %d %.17g\\n", info.steps, info.cuts, info.newton_iterations, info.t);',
        '  for (int k = 0; k < info.steps; ++k) printf("%.17g\\n", hist[k]);',
        f'  for (int k = 0; k < {8 * n}; ++k) printf("%.17g\\n", u[k]);',
        f'  for (int k = 0; k < {n}; ++k) printf("%.17g\\n", coke[k]);',
        "  isc_destroy(h);",
        "  return 0;",
        "}"]
    (tmp_path / "tube.c").write_text("\n".join(src) + "\n")
    libdir = os.path.join(ROOT, "paper_1811_11992_gb300", "_lib")
    exe = tmp_path / "tube"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(tmp_path / "tube.c"),
                    "-L", libdir, "-lisc", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    return exe, case


def test_c_program_compiles_against_the_header(tmp_path):
    """The generated program (every input structure filled field by field)
    compiles with -Wall -Werror and links against libisc.so, without a GPU."""
    exe, _ = _program(tmp_path)
    assert exe.exists()


@pytest.mark.gpu
def test_c_program_runs_the_time_loop_like_the_binding(tmp_path):
    from paper_1811_11992_gb300 import isc
    exe, case = _program(tmp_path)
    n = case.n
    t_end, dt0, dt_max = T_END, DT0, DT_MAX
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=600).stdout.split()
    steps, cuts, newton = int(out[0]), int(out[1]), int(out[2])
    t = float(out[3])
    vals = np.array([float(v) for v in out[4:]])
    dts_c, u_c, c_c = vals[:steps], vals[steps:steps + 8 * n].reshape(8, n), vals[steps + 8 * n:]

    sim = isc.Simulator(case, tol_newton=1e-6, maxit_newton=25, tol_lin=1e-12, maxit_lin=400)
    sim.init_equilibrium()
    info, dts = sim.run(t_end, dt0, dt_max)
    u_p, c_p = sim.get_state()
    sim.close()
    assert (steps, cuts, newton) == (info.steps, info.cuts, info.newton_iterations) and steps > 5
    assert t == info.t
    assert np.array_equal(dts_c, dts)
    assert np.array_equal(u_c, u_p) and np.array_equal(c_c, c_p)
