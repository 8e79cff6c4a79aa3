"""Every name a committed Python module reads is defined (assigned, imported
or built in): a static check that catches, on the CPU, a NameError in code
paths that only run on a GPU."""
import builtins
import glob
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(
    ["bench.py", "__graft_entry__.py"]
    + [os.path.relpath(p, ROOT) for pat in ("paper_1105_4002_gb300/*.py", "oracle/*.py",
                                             "synth/*.py", "tests/*.py")
       for p in glob.glob(os.path.join(ROOT, pat))])


def _free_globals(table, out):
    for sym in table.get_symbols():
        if sym.is_global() and sym.is_referenced() and not sym.is_assigned():
            out.add(sym.get_name())
    for child in table.get_children():
        _free_globals(child, out)


@pytest.mark.parametrize("path", FILES)
def test_module_reads_no_undefined_name(path):
    src = open(os.path.join(ROOT, path)).read()
    top = symtable.symtable(src, path, "exec")
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    free = set()
    for child in top.get_children():
        _free_globals(child, free)
    missing = sorted(n for n in free if n not in defined and not hasattr(builtins, n)
                     and n != "__file__")
    assert not missing, (path, missing)
