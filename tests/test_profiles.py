"""The committed profile summaries stay reproducible from committed files: every summary is a
short text file, every profile case it names exists, and every ncu command in it leaves the
GPU clocks alone (CPU only)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))


def test_profiles_are_short_text_summaries():
    assert PROFILES
    for p in PROFILES:
        assert os.path.splitext(p)[1] in (".md", ".txt"), p
        assert os.path.getsize(p) < 64 * 1024, p


def test_named_profile_cases_exist():
    from paper_2311_11943_gb300 import profile_cases
    named = set()
    for p in PROFILES:
        with open(p) as fh:
            named |= set(re.findall(r"profile_cases\s+(\w+)", fh.read()))
    assert named
    assert named <= set(profile_cases.CASES), sorted(named - set(profile_cases.CASES))


def test_every_ncu_command_keeps_the_clocks():
    for p in PROFILES:
        with open(p) as fh:
            text = fh.read()
        # commands sit in fenced blocks; one may span continuation lines
        for block in re.findall(r"```[^\n]*\n(.*?)```", text, flags=re.S):
            joined = re.sub(r"\\\s*\n\s*", " ", block)
            for line in joined.splitlines():
                if re.search(r"(^|[\s;&(])ncu\s", line):
                    assert "--clock-control none" in line, (p, line)
