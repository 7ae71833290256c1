"""The ncu summaries under profiles/ are short text files whose capture
commands run committed code only (bench.py) and leave the GPU clocks alone
(every capture command passes --clock-control none)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def commands(text):
    """The shell commands of a summary's indented code lines, continuation
    lines (ending in a backslash) joined."""
    out, cur = [], ""
    for line in text.splitlines():
        if not line.startswith("    "):
            if cur:
                out.append(cur)
            cur = ""
            continue
        part = line.strip()
        cur = (cur + " " + part.rstrip("\\").strip()) if cur else part.rstrip("\\").strip()
        if not part.endswith("\\"):
            out.append(cur)
            cur = ""
    if cur:
        out.append(cur)
    return out


def test_profiles_are_short_text_summaries():
    names = sorted(os.listdir(PROFILES))
    assert names, "no profile summaries"
    for n in names:
        assert os.path.splitext(n)[1] in (".md", ".txt"), n
        size = os.path.getsize(os.path.join(PROFILES, n))
        assert size < 16 * 1024, (n, size)


def test_capture_commands_leave_clocks_alone_and_run_committed_code():
    captures = 0
    for n in sorted(os.listdir(PROFILES)):
        text = open(os.path.join(PROFILES, n)).read()
        for cmd in commands(text):
            if not re.match(r"ncu\s", cmd) or re.match(r"ncu\s+-i\s", cmd):
                continue
            captures += 1
            assert "--clock-control none" in cmd, (n, cmd)
            assert "python bench.py" in cmd, (n, cmd)
            assert "_work" not in cmd, (n, cmd)
    assert captures >= 10
