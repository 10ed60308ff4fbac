"""Static checks of bench.py's GPU-only code paths (CPU, no GPU needed).

Most of bench.py runs only on a GPU, so a name that a function reads but
never binds would surface only there.  This walks each function of the
module and fails on a load of a name that is neither bound in the function
(arguments, assignments, imports, nested definitions) nor defined at module
level or a builtin.
"""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _module_names(tree):
    names = set(dir(builtins)) | {"__file__", "__name__"}
    for node in tree.body:
        if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(node.name)
            continue
        for n in ast.walk(node):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store):
                names.add(n.id)
            if isinstance(n, (ast.Import, ast.ImportFrom)):
                names.update((a.asname or a.name).split(".")[0] for a in n.names)
    return names


def _unbound_loads(fn, module_names):
    bound = set()
    for n in ast.walk(fn):
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            bound.add(n.id)
        elif isinstance(n, ast.arg):
            bound.add(n.arg)
        elif isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)) and n is not fn:
            bound.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            bound.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            bound.add(n.name)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            bound.update(n.names)
    return [(n.lineno, n.id) for n in ast.walk(fn)
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)
            and n.id not in bound and n.id not in module_names]


def unbound_names(path):
    tree = ast.parse(open(path).read())
    module_names = _module_names(tree)
    out = []
    for node in tree.body:
        fns = [node] if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef)) else (
            [m for m in node.body if isinstance(m, (ast.FunctionDef, ast.AsyncFunctionDef))]
            if isinstance(node, ast.ClassDef) else [])
        for fn in fns:
            out += [(fn.name, line, name) for line, name in _unbound_loads(fn, module_names)]
    return out


def test_the_checker_finds_a_name_read_before_any_binding():
    src = "import os\nX = 1\ndef f(a):\n    b = a + X\n    return b + c\n"
    tree = ast.parse(src)
    fn = tree.body[2]
    assert _unbound_loads(fn, _module_names(tree)) == [(5, "c")]


def test_bench_functions_read_only_names_they_or_the_module_bind():
    assert unbound_names(os.path.join(ROOT, "bench.py")) == []


def test_entry_point_functions_read_only_names_they_or_the_module_bind():
    assert unbound_names(os.path.join(ROOT, "__graft_entry__.py")) == []
