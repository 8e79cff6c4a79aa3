"""Rules on the committed sources, checked on the CPU:
- no source names one of the batched-copy runtime / driver calls that are
  closed on the GPUs this code runs on (a source that names one is refused
  for GPU runs);
- code and comments do not point into the working folder;
- no committed file sits in a top-level tools/ or scripts/ folder."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EXT = (".py", ".cu", ".cuh", ".h", ".c", ".cpp", ".sh")


def committed():
    try:
        out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True,
                             check=True).stdout.split()
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("not a git checkout")
    return out


def closed_calls():
    # spelled in pieces so that this file does not name them itself
    stem = ["cudaMemcpy", "cudaMemcpy3D", "cuMemcpy", "cuMemcpy3D"]
    return [s + "Batch" + "Async" for s in stem]


def test_no_source_names_a_closed_call():
    names = closed_calls()
    for f in committed():
        if f.endswith(EXT) or f.endswith(".txt"):
            text = open(os.path.join(ROOT, f), errors="replace").read()
            for n in names:
                assert n not in text, (f, n)


def test_code_does_not_point_into_the_working_folder():
    marker = "_" + "work/"
    for f in committed():
        if f.endswith(EXT) and not f.startswith("tests/"):
            assert marker not in open(os.path.join(ROOT, f), errors="replace").read(), f


def test_no_top_level_tools_or_scripts_folder():
    assert not [f for f in committed() if f.split("/")[0] in ("tools", "scripts")]
