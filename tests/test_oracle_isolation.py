"""The oracle stays test infrastructure: the product package never imports it
(nor it the package), bench.py imports it only inside its CPU legs (the CPU
baseline and the reference arm) and __graft_entry__ only inside smoke()."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _oracle_imports(path):
    """(enclosing function name or None, line) of every import of oracle."""
    tree = ast.parse(open(path).read())
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append((func, child.lineno))
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.append((func, child.lineno))
            visit(child, f)
    visit(tree, None)
    return found


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2404_00774_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            assert _oracle_imports(os.path.join(pkg, name)) == [], name


def test_oracle_never_imports_the_product_package():
    odir = os.path.join(ROOT, "oracle")
    for name in os.listdir(odir):
        if not name.endswith(".py"):
            continue
        for node in ast.walk(ast.parse(open(os.path.join(odir, name)).read())):
            mods = [a.name for a in node.names] if isinstance(node, ast.Import) else \
                [node.module or ""] if isinstance(node, ast.ImportFrom) else []
            assert not any(m.split(".")[0] in ("paper_2404_00774_gb300", "torch") for m in mods), (name, mods)


def test_bench_imports_the_oracle_only_in_its_cpu_legs():
    sites = _oracle_imports(os.path.join(ROOT, "bench.py"))
    assert sites and {f for f, _ in sites} <= {"oracle_index", "time_oracle", "run_reference"}, sites


def test_entry_module_imports_the_oracle_only_in_smoke():
    sites = _oracle_imports(os.path.join(ROOT, "__graft_entry__.py"))
    assert sites and {f for f, _ in sites} == {"smoke"}, sites
