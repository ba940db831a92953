"""The commands recorded in profiles/*.md still run against the committed
tree: every `python bench.py ...` line parses with bench.py's own argument
parser, every `ncu -k regex:...` names a kernel that the CUDA sources define,
every `ncu` line passes `--clock-control none`, and no command reaches
outside the committed files."""
import re
import shlex
from pathlib import Path

import pytest

import bench

ROOT = Path(__file__).resolve().parent.parent
PROFILES = sorted((ROOT / "profiles").glob("*.md"))
CSRC = ROOT / "paper_2203_09087_gb300" / "csrc"


def _command_lines(text: str):
    """Indented command blocks with their backslash continuations joined."""
    out, cur = [], ""
    for line in text.splitlines():
        if not line.startswith("    "):
            if cur:
                out.append(cur)
            cur = ""
            continue
        piece = line.strip()
        if piece.endswith("\\"):
            cur += piece[:-1] + " "
        else:
            out.append(cur + piece)
            cur = ""
    if cur:
        out.append(cur)
    return [c for c in out if "python " in c or "ncu " in c]


def _strip_launch_bounds(decl: str) -> str:
    i = decl.find("__launch_bounds__")
    while i >= 0:
        j, depth = decl.index("(", i), 0
        for k in range(j, len(decl)):
            depth += {"(": 1, ")": -1}.get(decl[k], 0)
            if depth == 0:
                break
        decl = decl[:i] + decl[k + 1:]
        i = decl.find("__launch_bounds__")
    return decl


def _kernel_names():
    names = set()
    for f in list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")):
        text = f.read_text()
        for m in re.finditer(r"__global__", text):
            end = min(x for x in (text.find("{", m.end()), text.find(";", m.end()), len(text)) if x >= 0)
            decl = _strip_launch_bounds(text[m.end():end])
            hit = re.search(r"(\w+)\s*\(", decl)
            if hit:
                names.add(hit.group(1))
    return names


def _bench_invocations(cmd: str):
    for m in re.finditer(r"python bench\.py([^>|&]*)", cmd):
        yield shlex.split(m.group(1))


def test_every_profile_gives_its_command():
    assert PROFILES
    for p in PROFILES:
        assert _command_lines(p.read_text()), p.name


@pytest.mark.parametrize("path", PROFILES, ids=[p.name for p in PROFILES])
def test_recorded_commands_run_committed_files(path):
    kernels = _kernel_names()
    parser = bench.arg_parser()
    for cmd in _command_lines(path.read_text()):
        assert "_work" not in cmd, cmd
        for py in re.findall(r"python (\S+\.py)", cmd):
            assert (ROOT / py).is_file(), (path.name, py)
        for argv in _bench_invocations(cmd):
            parser.parse_args(argv)  # exits (SystemExit) on a flag bench.py no longer has
        if "ncu " in cmd:
            assert "--clock-control none" in cmd, (path.name, cmd)
            for pat in re.findall(r"-k regex:(\S+)", cmd):
                assert any(re.search(pat, k) for k in kernels), (path.name, pat)


def test_kernel_name_scan_finds_the_hot_kernels():
    names = _kernel_names()
    for k in ["bs3_kernel", "bs2d_kernel", "batch_kernel", "scan_kernel", "collect_kernel"]:
        assert k in names, k
