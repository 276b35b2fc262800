"""bench.py's GPU-only paths (--mixed, --ess, --batch, ...) cannot run on the
CPU, so a name used but bound nowhere would surface only on a GPU machine: check
statically that every name a function of bench.py loads is a parameter or
local of it or of an enclosing function, a module-level name, or a builtin."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bound(node):
    names = set()
    for sub in ast.walk(node):
        if isinstance(sub, ast.Name) and isinstance(sub.ctx, (ast.Store, ast.Del)):
            names.add(sub.id)
        elif isinstance(sub, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(sub.name)
        elif isinstance(sub, ast.arg):
            names.add(sub.arg)
        elif isinstance(sub, ast.alias):
            names.add((sub.asname or sub.name).split(".")[0])
        elif isinstance(sub, ast.ExceptHandler) and sub.name:
            names.add(sub.name)
    return names


def test_every_loaded_name_is_bound():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    module_names = _bound(ast.Module(body=[n for n in tree.body if not isinstance(n, ast.FunctionDef)],
                                     type_ignores=[])) | {n.name for n in tree.body if isinstance(n, ast.FunctionDef)}
    known = module_names | set(dir(builtins))
    missing = []

    # each top-level function with everything bound anywhere inside it (its
    # closures see their enclosing function's names)
    for fn in tree.body:
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            scope = known | _bound(fn)
            for sub in ast.walk(fn):
                if isinstance(sub, ast.Name) and isinstance(sub.ctx, ast.Load) and sub.id not in scope:
                    missing.append((fn.name, sub.id, sub.lineno))
    assert not missing, missing
