"""Every command a profile summary names runs committed files only.

Each summary under profiles/ states the command that produced it. These
checks parse every `python bench.py ...` command with the benchmark's own
argument parser, and require every ncu command to use --clock-control none
and to profile a bench.py command.
"""
import glob
import os
import re
import shlex
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(path):
    """Commands in indented code blocks, and inline `python bench.py ...`."""
    text = open(path).read().replace("\\\n", " ")
    cmds = [line.strip() for line in text.splitlines()
            if line.startswith("    ") and line.strip().startswith(("ncu ", "python "))]
    cmds += re.findall(r"`(python bench\.py[^`]*)`", text)
    return [re.sub(r"\s+", " ", c) for c in cmds]


def test_profiles_exist():
    assert PROFILES


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_bench_commands_parse(path, monkeypatch):
    for cmd in _commands(path):
        if "bench.py" not in cmd:
            continue
        argv = shlex.split(cmd[cmd.index("bench.py"):])
        # `--workload a|b|c` names several commands at once
        alts = [argv]
        for i, tok in enumerate(argv):
            if "|" in tok:
                alts = [argv[:i] + [choice] + argv[i + 1:] for choice in tok.split("|")]
        for a in alts:
            monkeypatch.setattr(sys, "argv", a)
            bench.parse()  # exits (SystemExit) on an unknown option or workload


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_ncu_commands_leave_clocks_alone(path):
    for cmd in _commands(path):
        if cmd.startswith("ncu "):
            assert "--clock-control none" in cmd, cmd
            assert "bench.py" in cmd, cmd
