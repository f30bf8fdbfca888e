"""The committed profile summaries keep their rules (CPU): short text files only, each
with the full command that made it; every ncu command leaves the clocks alone
(`--clock-control none`); every command runs committed files only, and the benchmark
arguments it records still parse with the benchmark's own parser."""
import json
import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def commands(text):
    """Logical command lines of the fenced blocks (backslash continuations joined,
    comments and output redirections removed), split at `&&`."""
    out = []
    for block in re.findall(r"```[a-z]*\n(.*?)```", text, re.S):
        joined = re.sub(r"\\\n\s*", " ", block)
        for line in joined.splitlines():
            line = line.split("#", 1)[0].strip()
            for part in line.split("&&"):
                part = re.sub(r"\s*>\s*\S+\s*$", "", part.strip())
                if part:
                    out.append(part)
    return out


def test_profiles_are_short_text_with_commands():
    files = sorted(os.listdir(PROF))
    assert files and any(f.startswith("launches_") for f in files)
    for f in files:
        path = os.path.join(PROF, f)
        assert f.endswith((".md", ".txt", ".json")), f
        assert os.path.getsize(path) < 16 * 1024, f
        if f.endswith(".json"):
            rec = json.load(open(path))
            assert os.path.exists(os.path.join(ROOT, rec["capture"])), f
            continue
        cmds = commands(open(path).read())
        assert any(c.startswith("ncu ") for c in cmds), "%s gives no ncu command" % f


def test_recorded_commands_run_committed_files_and_parse():
    sys.path.insert(0, ROOT)
    import bench
    n = 0
    for f in sorted(os.listdir(PROF)):
        if not f.endswith(".md"):
            continue
        for c in commands(open(os.path.join(PROF, f)).read()):
            assert "_work" not in c and "/root/" not in c, (f, c)
            argv = shlex.split(c)
            if argv[0] == "ncu":
                assert "--clock-control" in argv and argv[argv.index("--clock-control") + 1] == "none", (f, c)
                argv = argv[argv.index("python"):]
            if argv[0] != "python":
                continue
            script = argv[1]
            assert os.path.exists(os.path.join(ROOT, script)), (f, script)
            if script == "bench.py":
                args = bench.parse_args(argv[2:])
                assert args.workload in bench.WORKLOADS
                n += 1
    assert n >= 8
