"""The committed ncu summaries under profiles/ name the command that made
them, and that command runs committed files only, with the clocks left alone
(--clock-control none on every ncu line)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_summary_commands_run_committed_files(path):
    text = open(path).read()
    scripts = re.findall(r"\bpython3?\s+(\S+\.py)\b", text)
    assert scripts, "a summary gives the command that made it"
    for s in scripts:
        assert not s.startswith("_work") and "/_work/" not in s, s
        assert os.path.exists(os.path.join(ROOT, s)), s
    commands = [line for line in text.splitlines() if re.match(r"\s{4,}ncu\s", line)]
    assert commands, "a summary gives the ncu command"
    for line in commands:
        assert "--clock-control none" in line, line


def test_traffic_record_names_existing_sources():
    import json
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic_64cubed.json")))
    for name in rec["kernel_sources"]:
        assert os.path.exists(os.path.join(ROOT, name)), name
    assert rec["config"] == "c64" and rec["storage"] == "fp32"
