"""The ncu summaries under profiles/ are short text files whose commands run committed code only: every
module, script and package attribute they name exists in the repository."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def _files():
    return sorted(f for f in os.listdir(PROF) if not f.startswith("."))


def test_profiles_are_short_text():
    for f in _files():
        assert f.endswith((".md", ".txt")), f
        assert os.path.getsize(os.path.join(PROF, f)) < 16 * 1024, f


def test_profile_commands_name_committed_code():
    for f in _files():
        text = open(os.path.join(PROF, f)).read()
        assert "_work" not in text and "/root/" not in text, f
        for mod in re.findall(r"python -m ([A-Za-z0-9_.]+)", text):
            assert importlib.util.find_spec(mod) is not None, (f, mod)
        for script in re.findall(r"python ([A-Za-z0-9_./]+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), (f, script)
        for names in re.findall(r"from paper_1307_6748_gb300 import ([a-z_, ]+)", text):
            for n in (x.strip() for x in names.split(",")):
                assert os.path.exists(os.path.join(ROOT, "paper_1307_6748_gb300", n + ".py")), (f, n)
        # the package attributes a command calls exist (isis.X, synth.X)
        from paper_1307_6748_gb300 import isis, synth
        for mod, name in re.findall(r"\b(isis|synth)\.([A-Za-z_][A-Za-z0-9_]*)", text):
            assert hasattr({"isis": isis, "synth": synth}[mod], name), (f, mod, name)
