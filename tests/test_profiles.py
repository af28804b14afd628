"""The committed profile summaries are reproducible from committed files: every
command they give runs scripts of this repository (not scratch files), every
ncu invocation leaves the GPU clocks alone, and they hold text only."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def _tracked():
    out = subprocess.check_output(["git", "ls-files"], cwd=ROOT, text=True)
    return set(out.split())


def _code_blocks(text):
    return re.findall(r"```[a-z]*\n(.*?)```", text, flags=re.S)


def test_profiles_hold_short_text_only():
    for f in os.listdir(PROF):
        assert f.endswith((".md", ".txt", ".json")), f
        assert os.path.getsize(os.path.join(PROF, f)) < 64 * 1024, f


def test_profile_commands_run_committed_files_and_keep_clocks():
    tracked = _tracked()
    n_ncu = 0
    for f in sorted(os.listdir(PROF)):
        if not f.endswith(".md"):
            continue
        for block in _code_blocks(open(os.path.join(PROF, f)).read()):
            cmd = block.replace("\\\n", " ")
            for script in re.findall(r"python3?\s+([\w./-]+\.py)", cmd):
                assert not script.startswith("_work"), (f, script)
                assert script in tracked, (f, script)
            for line in cmd.splitlines():
                if re.search(r"(^|\s)ncu\s", line):
                    n_ncu += 1
                    assert "--clock-control none" in line, (f, line)
    assert n_ncu >= 4


def test_no_committed_code_uses_scratch_files():
    """Scratch work (probes, sweeps, notes) lives in an ignored folder that no
    committed file imports, reads or runs."""
    # the folder name on its own (not inside identifiers such as a workspace)
    scratch = re.compile(r"(?<![\w])_" + r"work\b")
    for f in _tracked():
        if f.endswith(".md") or f == ".gitignore" or not os.path.isfile(os.path.join(ROOT, f)):
            continue
        if f == "tests/test_profiles.py":
            continue
        text = open(os.path.join(ROOT, f), errors="replace").read()
        assert not scratch.search(text), f
