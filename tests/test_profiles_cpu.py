"""The committed ncu summaries stay reproducible: each gives its ncu command
with --clock-control none (or points to the summary that holds it), every
`python bench.py ...` line in them still parses with the benchmark's
current arguments, and profiles/traffic.json names files that exist."""

import glob
import json
import os
import re
import shlex
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(text):
    """Shell commands in the fenced blocks, continuation lines joined."""
    out = []
    for block in re.findall(r"```[a-z]*\n(.*?)```", text, flags=re.S):
        out.extend(c.strip() for c in block.replace("\\\n", " ").splitlines() if c.strip())
    return out


def test_there_are_summaries():
    assert len(SUMMARIES) >= 4


@pytest.mark.parametrize("path", SUMMARIES, ids=os.path.basename)
def test_summary_gives_its_ncu_command(path):
    text = open(path).read()
    cmds = [c for c in _commands(text) if c.startswith("ncu ")]
    if not cmds:
        refs = re.findall(r"`([a-z0-9_]+\.md)`", text)
        assert refs and all(os.path.exists(os.path.join(ROOT, "profiles", r)) for r in refs), path
        return
    for c in cmds:
        assert "--clock-control none" in c, c


@pytest.mark.parametrize("path", SUMMARIES, ids=os.path.basename)
def test_bench_lines_parse_with_the_current_arguments(path, monkeypatch):
    for c in _commands(open(path).read()):
        if "python bench.py" not in c:
            continue
        argv = shlex.split(c.split("python bench.py", 1)[1])
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        args = bench.parse()
        assert args.impl in ("ours", "reference")


def test_traffic_record_names_existing_files():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for name, ent in rec.items():
        assert os.path.exists(os.path.join(ROOT, ent["source"])), ent["source"]
        for k in ent["kernel_files"]:
            assert os.path.exists(os.path.join(ROOT, k)), k
