"""The committed ncu summaries in profiles/ against the sources and the bench (no GPU): bench.py
reports a kernel's DRAM traffic only from a summary taken on the current kernel sources (null
otherwise), and every bench command that a summary gives as the one that made it is a valid
bench.py command line."""
import os
import re
import shlex

import pytest

import bench

PROFILES = os.path.join(bench.ROOT, "profiles")


def summaries():
    return sorted(f for f in os.listdir(PROFILES) if f.endswith((".md", ".txt")))


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_PROFILES))
def test_kernel_traffic_only_from_current_sources(kernel):
    txt = open(os.path.join(PROFILES, bench.KERNEL_PROFILES[kernel][0])).read()
    sha = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    assert sha, "summary without source_sha256"
    if sha.group(1) == bench.kernel_source_sha(kernel):
        assert bench.profiled_traffic(kernel) > 0
    else:                                   # taken on other sources: the bench reports null
        assert bench.profiled_traffic(kernel) is None


def bench_commands(txt):
    """Every 'python bench.py ...' command of a summary, line continuations joined."""
    joined = re.sub(r"\\\n\s*", " ", txt)
    return [shlex.split(m) for m in re.findall(r"python bench\.py([^\n`]*)", joined)]


@pytest.mark.parametrize("name", summaries())
def test_summary_gives_valid_bench_commands(name):
    txt = open(os.path.join(PROFILES, name)).read()
    cmds = bench_commands(txt)
    assert cmds, f"{name} gives no bench command"
    ap = bench.build_parser()
    for argv in cmds:
        ap.parse_args(argv)                     # exits (fails the test) on an unknown option
    for line in re.sub(r"\\\n\s*", " ", txt).splitlines():
        if line.strip().startswith("ncu ") and "-i " not in line:
            assert "--clock-control none" in line, f"{name}: ncu without --clock-control none"
