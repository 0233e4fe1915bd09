"""The commands quoted in profiles/ run committed files only: every
`python bench.py ...` line there parses with bench.py's own arguments, and
every Python file a command names exists in the repository and is not
ignored by git (so a reader can rerun it from a checkout)."""
import os
import shlex
import subprocess
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


def _ignored(path):
    if not os.path.isdir(os.path.join(ROOT, ".git")):
        return False
    r = subprocess.run(["git", "-C", ROOT, "check-ignore", "-q", path],
                       capture_output=True)
    return r.returncode == 0


def test_profile_commands_parse_with_bench_arguments(monkeypatch):
    cmds = _commands()
    assert cmds, "no bench command quoted in profiles/"
    for fn, line in cmds:
        toks = shlex.split(line.replace("`", " "))
        for t in toks:
            if t.endswith(".py"):
                assert os.path.exists(os.path.join(ROOT, t)), (fn, t)
                assert not _ignored(t), (fn, t)
        bt = shlex.split(line[line.index("bench.py"):].replace("`", " "))
        monkeypatch.setattr(sys, "argv", ["bench.py"] + bt[1:])
        bench.parse_args()                      # SystemExit on an unknown flag
