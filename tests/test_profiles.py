"""The ncu summaries under profiles/ name the commands that produced them;
those commands must still run on the committed files: every `bench.py`
invocation parses with bench.py's own argument parser, every `ncu` command
leaves the GPU clocks alone (`--clock-control none`), and all of them write
their reports into one scratch folder that .gitignore keeps out of the
repository (raw reports are not committed)."""
import glob
import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def commands(text):
    """Shell commands in the indented blocks of a summary, with their
    backslash continuations joined."""
    out, cur = [], ""
    for line in text.splitlines():
        if not line.startswith("    "):
            if cur:
                out.append(cur)
            cur = ""
            continue
        body = line.strip()
        cur = (cur + " " + body[:-1].strip()) if body.endswith("\\") else (cur + " " + body)
        if not body.endswith("\\"):
            out.append(cur.strip())
            cur = ""
    if cur:
        out.append(cur.strip())
    return [c for c in out if c.startswith(("ncu ", "python "))]


def test_profile_commands_run_committed_files():
    sys.path.insert(0, ROOT)
    import bench
    parser = bench.make_parser()
    summaries = glob.glob(os.path.join(ROOT, "profiles", "*.md"))
    assert summaries
    seen_bench = 0
    out_dirs = set()
    for path in summaries:
        cmds = commands(open(path).read())
        assert cmds, f"{os.path.basename(path)} names no command"
        for cmd in cmds:
            argv = shlex.split(cmd)
            if argv[0] == "ncu":
                assert "--clock-control" in argv and \
                    argv[argv.index("--clock-control") + 1] == "none", cmd
                for flag in ("-o", "--log-file"):
                    if flag in argv:
                        out = argv[argv.index(flag) + 1]
                        assert "/" in out and not os.path.isabs(out), cmd
                        out_dirs.add(out.split("/")[0])
            if "bench.py" in argv:
                rest = argv[argv.index("bench.py") + 1:]
                parser.parse_args(rest)  # exits on an unknown flag or value
                seen_bench += 1
            for word in argv:
                if word.endswith(".py"):
                    assert os.path.exists(os.path.join(ROOT, word)), (word, cmd)
                assert not re.search(r"_work/", word), cmd
    assert seen_bench > 0
    assert len(out_dirs) == 1, out_dirs
    ignored = [line.strip().strip("/") for line in open(os.path.join(ROOT, ".gitignore"))]
    assert out_dirs.pop() in ignored
