"""The ncu summaries under profiles/ give the commands that made them: every
`python bench.py ...` in them parses with bench.py's own arguments, every
ncu command leaves the clocks alone (`--clock-control none`) and names one
kernel or only the launch time, and nothing runs a file outside the
repository's committed tree."""
import glob
import os
import re
import shlex

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands():
    """(file, command) for every command line in the fenced blocks, with
    backslash continuations joined and shell loops reduced to their body."""
    out = []
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(f).read()
        for block in re.findall(r"```[a-z]*\n(.*?)```", text, flags=re.S):
            joined = re.sub(r"\\\n\s*", " ", block)
            for line in joined.splitlines():
                line = line.strip()
                if not line or line.startswith(("for ", "done")):
                    continue
                out.append((os.path.basename(f), line.rstrip(";")))
    return out


def test_every_summary_has_commands():
    files = sorted(os.path.basename(f) for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    have = {f for f, _ in _commands()}
    assert have == set(files), set(files) - have


def test_bench_arguments_parse():
    ap = bench.build_parser()
    n = 0
    for f, cmd in _commands():
        words = shlex.split(cmd.replace("$k", "k_ilu"))
        if "bench.py" not in words:
            continue
        i = words.index("bench.py")
        assert words[i - 1] == "python", (f, cmd)
        args = ap.parse_args(words[i + 1:])            # exits (fails) on an unknown flag
        assert args.profile_step > 0 or args.profile_dense > 0, (f, cmd)
        n += 1
    assert n >= 8


def test_ncu_commands_leave_clocks_alone():
    for f, cmd in _commands():
        words = shlex.split(cmd.replace("$k", "k_ilu"))
        if not words or words[0] != "ncu":
            continue
        assert "--clock-control" in words and words[words.index("--clock-control") + 1] == "none", (f, cmd)
        if "--set" in words:                           # a full capture: one kernel, a few launches
            assert "-k" in words and "-c" in words, (f, cmd)
            assert int(words[words.index("-c") + 1]) <= 3, (f, cmd)
        else:
            assert "--metrics" in words, (f, cmd)


def test_commands_run_committed_files_only():
    for f, cmd in _commands():
        assert "_work" not in cmd and "/root" not in cmd, (f, cmd)
        for w in shlex.split(cmd.replace("$k", "k_ilu")):
            if w.endswith(".py"):
                assert os.path.exists(os.path.join(ROOT, w)), (f, w)


def test_referenced_summaries_exist():
    """Every profiles/*.md that the README, the design notes or bench.py names exists."""
    for path in [os.path.join(ROOT, f) for f in ("README.md", "DESIGN.md", "bench.py")]:
        for ref in re.findall(r"profiles/[A-Za-z0-9_.-]+\.md", open(path).read()):
            assert os.path.exists(os.path.join(ROOT, ref)), (os.path.basename(path), ref)
