"""bench.py's runners build their JSON lines from many locals; a name used in
one runner but defined only in another fails only when that workload runs on a
GPU.  This check (CPU, no import of the module) finds, in every function, the
names it loads that are neither bound in it (arguments, assignments, loops,
imports, nested definitions, comprehension and exception targets), nor at
module level, nor builtins."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _module_names(tree):
    names = set()
    for node in tree.body:
        if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(node.name)
        elif isinstance(node, (ast.Assign, ast.AnnAssign, ast.AugAssign)):
            targets = node.targets if isinstance(node, ast.Assign) else [node.target]
            for t in targets:
                names.update(n.id for n in ast.walk(t) if isinstance(n, ast.Name))
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            names.update((a.asname or a.name).split(".")[0] for a in node.names)
    return names


def _bound_in(fn):
    bound = set()
    for node in ast.walk(fn):
        if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.Lambda)):
            if node is not fn and not isinstance(node, ast.Lambda):
                bound.add(node.name)
            a = node.args
            for arg in a.posonlyargs + a.args + a.kwonlyargs:
                bound.add(arg.arg)
            if a.vararg:
                bound.add(a.vararg.arg)
            if a.kwarg:
                bound.add(a.kwarg.arg)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
            bound.add(node.id)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            bound.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            bound.add(node.name)
        elif isinstance(node, (ast.Global, ast.Nonlocal)):
            bound.update(node.names)
    return bound


def test_bench_functions_use_only_defined_names():
    src = open(os.path.join(ROOT, "bench.py")).read()
    tree = ast.parse(src)
    module = _module_names(tree)
    problems = []
    for fn in tree.body:
        if not isinstance(fn, ast.FunctionDef):
            continue
        bound = _bound_in(fn)
        for node in ast.walk(fn):
            if isinstance(node, ast.Name) and isinstance(node.ctx, ast.Load):
                if node.id not in bound and node.id not in module and not hasattr(builtins, node.id):
                    problems.append(f"{fn.name}: {node.id} (line {node.lineno})")
    assert not problems, problems
