"""The profile summaries are short text, each with the command that made it, and
those commands run files that are in the repository."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _summaries():
    return sorted(f for f in os.listdir(PROFILES) if not f.startswith("."))


def test_profiles_are_short_text_summaries():
    names = _summaries()
    assert names
    for f in names:
        assert f.endswith((".md", ".txt")), f
        assert os.path.getsize(os.path.join(PROFILES, f)) < 16 * 1024, f


def test_each_summary_gives_its_commands_and_they_run_committed_files():
    for f in _summaries():
        text = open(os.path.join(PROFILES, f)).read()
        blocks = re.findall(r"```\n(.*?)```", text, flags=re.S)
        cmds = [b for b in blocks if re.search(r"\b(python|nvcc|ncu)\b", b)]
        assert cmds, f"{f}: no command"
        for b in cmds:
            for path in re.findall(r"[\w./-]+\.(?:py|cu|c|h|sh)\b", b):
                if path.startswith("gpurun_out/"):
                    continue          # outputs of the command, not inputs
                assert os.path.exists(os.path.join(ROOT, path)), f"{f}: {path} is not in the repository"
