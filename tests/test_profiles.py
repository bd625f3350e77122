"""The profile summaries give the commands that produced them; every
`python bench.py ...` command there must still parse with the benchmark's
current options (so the recorded captures stay reproducible)."""
import glob
import os
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands():
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")          # join continued lines
        for line in text.splitlines():
            if "python bench.py" in line:
                out.append((os.path.basename(path), line.split("python bench.py", 1)[1]))
    return out


def test_profiles_name_their_commands():
    files = {f for f, _ in _commands()}
    assert files == {os.path.basename(p) for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))}


@pytest.mark.parametrize("name,argv", _commands())
def test_profile_command_parses(name, argv):
    sys.path.insert(0, ROOT)
    import bench
    bench._parser().parse_args(shlex.split(argv))
