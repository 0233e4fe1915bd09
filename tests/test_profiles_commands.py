"""The commands quoted in profiles/ run committed files only: every
`python bench.py ...` line there parses with bench.py's own arguments, and
no command names a working-file folder."""
import os
import re
import shlex
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands():
    out = []
    for fn in sorted(os.listdir(PROFILES)):
        if not fn.endswith((".md", ".txt")):
            continue
        text = open(os.path.join(PROFILES, fn)).read().replace("\\\n", " ")
        for line in text.splitlines():
            if "bench.py" in line and "python" in line:
                out.append((fn, line.strip()))
    return out


def test_profile_commands_parse_with_bench_arguments(monkeypatch):
    cmds = _commands()
    assert cmds, "no bench command quoted in profiles/"
    for fn, line in cmds:
        assert "_work" not in line and "gpurun_out/" not in line.split("bench.py")[1], (fn, line)
        toks = shlex.split(line[line.index("bench.py"):])
        args = [t for t in toks[1:] if not t.startswith("`")]
        monkeypatch.setattr(sys, "argv", ["bench.py"] + args)
        bench.parse_args()                      # SystemExit on an unknown flag
