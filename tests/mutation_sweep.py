"""Mutation sweep of the oracle's pins (CPU only; not collected by pytest).

Plants one small mistake at a time in a copy of one ``oracle/`` module -- an
arithmetic operator swapped (+ <-> -, * <-> /), a unary minus dropped, a
comparison made strict or non-strict, a numeric literal changed (an integer
by +1, a float by x1.25) -- and runs the CPU pins (``tests/test_oracle_*.py``,
first failure stops) on that copy. A mutant the pins reject is "killed"; one
they accept "survived" and is either equivalent (it changes no result the
method defines: a default argument every caller overrides, an initial value the
first iteration overwrites, a tie in a strict/non-strict test that real data
never meets) or a gap in the pins.

    python tests/mutation_sweep.py --module linalg --jobs 8 --out sweep.jsonl
    python tests/mutation_sweep.py --module linalg --only-survivors sweep.jsonl --out again.jsonl

Each line of the output names the module, the mutant's index and line, what
was changed, and the pytest exit status (0 = survived).
"""
import argparse
import ast
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# fastest pins first, so that most mutants die within seconds
PINS = ["test_oracle_props.py", "test_oracle_transport.py", "test_oracle_residual.py", "test_oracle_linalg.py", "test_oracle_wells.py",
        "test_oracle_cpr.py", "test_oracle_newton.py", "test_oracle_adjoint.py", "test_oracle_adjoint_wells.py"]
# each module's own pins run first
OWN = {"linalg": ["test_oracle_linalg.py"], "cpr": ["test_oracle_cpr.py"], "sim": ["test_oracle_newton.py"],
       "adjoint": ["test_oracle_adjoint.py", "test_oracle_adjoint_wells.py"]}
SWAP = {ast.Add: ast.Sub, ast.Sub: ast.Add, ast.Mult: ast.Div, ast.Div: ast.Mult}
CMP = {ast.Lt: ast.LtE, ast.LtE: ast.Lt, ast.Gt: ast.GtE, ast.GtE: ast.Gt}


def _sites(tree):
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.BinOp) and type(node.op) in SWAP:
            out.append((node, "binop"))
        elif isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.USub):
            out.append((node, "neg"))
        elif isinstance(node, ast.Compare) and len(node.ops) == 1 and type(node.ops[0]) in CMP:
            out.append((node, "cmp"))
        elif isinstance(node, ast.Constant) and type(node.value) in (int, float):
            out.append((node, "const"))
    return out


class _Plant(ast.NodeTransformer):
    def __init__(self, target, kind):
        self.target, self.kind, self.desc = target, kind, None

    def visit(self, node):
        if node is not self.target:
            return super().visit(node)
        if self.kind == "binop":
            node.op = SWAP[type(node.op)]()
            self.desc = "operator -> " + type(node.op).__name__
            return node
        if self.kind == "neg":
            self.desc = "unary minus dropped"
            return node.operand
        if self.kind == "cmp":
            node.ops = [CMP[type(node.ops[0])]()]
            self.desc = "comparison -> " + type(node.ops[0]).__name__
            return node
        v = node.value
        nv = v + 1 if isinstance(v, int) else (v * 1.25 if v != 0 else 1e-3)
        self.desc = f"literal {v!r} -> {nv!r}"
        return ast.copy_location(ast.Constant(nv), node)


def mutants(module):
    src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
    n = len(_sites(ast.parse(src)))
    for i in range(n):
        tree = ast.parse(src)
        node, kind = _sites(tree)[i]
        plant = _Plant(node, kind)
        tree = ast.fix_missing_locations(plant.visit(tree))
        yield dict(module=module, idx=i, line=node.lineno, kind=kind, desc=plant.desc, code=ast.unparse(tree))


def run_one(m, timeout, workdir):
    os.makedirs(workdir, exist_ok=True)
    work = tempfile.mkdtemp(prefix="mutant_", dir=workdir)
    try:
        for d in ("tests", "isc_inputs", "oracle"):
            shutil.copytree(os.path.join(ROOT, d), os.path.join(work, d),
                            ignore=shutil.ignore_patterns("__pycache__", "golden_out*"))
        with open(os.path.join(work, "oracle", m["module"] + ".py"), "w") as f:
            f.write(m["code"])
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
        cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
        own = OWN.get(m["module"], [])
        cmd += [os.path.join("tests", p) for p in own + [q for q in PINS if q not in own]]
        t0 = time.time()
        try:
            p = subprocess.run(cmd, cwd=work, capture_output=True, text=True, env=env, timeout=timeout)
            rc, out = p.returncode, p.stdout
        except subprocess.TimeoutExpired:
            rc, out = -1, ""                         # a mutant that loops: killed by the clock
        failed = [ln for ln in out.splitlines() if ln.startswith(("FAILED", "ERROR"))]
        return dict(module=m["module"], idx=m["idx"], line=m["line"], kind=m["kind"], desc=m["desc"], rc=rc,
                    secs=round(time.time() - t0, 1), killed_by=failed[:1])
    finally:
        shutil.rmtree(work, ignore_errors=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--module", required=True, help="oracle module name, e.g. linalg")
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--timeout", type=float, default=600.0)
    ap.add_argument("--only-survivors", help="a previous output: rerun only the mutants that survived there")
    ap.add_argument("--workdir", default=os.path.join(ROOT, ".mutation_work"),
                    help="where the mutated copies live while their pins run (removed after each)")
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    ms = list(mutants(a.module))
    if a.only_survivors:
        keep = {r["idx"] for r in map(json.loads, open(a.only_survivors)) if r["rc"] == 0 and r["module"] == a.module}
        ms = [m for m in ms if m["idx"] in keep]
    killed = survived = 0
    with open(a.out, "w") as fo, ThreadPoolExecutor(a.jobs) as ex:
        for r in ex.map(lambda m: run_one(m, a.timeout, a.workdir), ms):
            fo.write(json.dumps(r) + "\n")
            fo.flush()
            killed += r["rc"] != 0
            survived += r["rc"] == 0
    print(json.dumps(dict(module=a.module, mutants=len(ms), killed=killed, survived=survived)))


if __name__ == "__main__":
    main()
