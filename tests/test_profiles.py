"""The committed ncu summaries against the sources they describe: bench.py
reports an event kernel's DRAM traffic only from a summary whose source
digest matches the kernel sources, so a kernel change without a new capture
would silently turn `roofline.traffic` into null.  Also: every summary
gives the command that made it, and that command runs committed files."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_event_kernel_summaries_match_the_sources():
    for workload in ("prod3_1e8_f32", "decay_1e7"):
        traffic = bench.profiled_traffic(workload)
        assert traffic is not None, f"profiles/{workload}_events_ff.md does not match the kernel sources"
        # the columns once (12 or 8 bytes per event) plus a few per cent of records and tree
        n, width = (1e8, 12) if workload == "prod3_1e8_f32" else (1e7, 8)
        assert n * width <= traffic <= 1.05 * n * width


def test_every_summary_gives_its_command():
    names = [f for f in os.listdir(PROFILES) if f.endswith((".md", ".txt"))]
    assert names
    for name in names:
        text = open(os.path.join(PROFILES, name)).read()
        cmds = re.findall(r"^\s+(?:python|ncu)\b.*$", text, re.M)
        assert cmds, f"{name}: no command line"
        for c in cmds:
            assert "_work/" not in c and "/root/" not in c, f"{name}: {c.strip()}"
        for script in re.findall(r"python (?:-m pytest )?(\S+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), f"{name}: {script} is not committed"
