"""The committed profile summaries: short text only, each naming the command that made it,
every ncu command leaving the GPU clocks alone, and every command running files of this
repository.  profiles/traffic.json names workloads and kernel classes that bench.py knows."""
import glob
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands(text):
    return [line.strip() for line in text.splitlines() if line.strip().startswith("ncu ")]


def _check_command(cmd):
    assert "--clock-control none" in cmd, cmd
    m = re.search(r"\bpython\s+(\S+)", cmd)
    assert m, cmd
    assert os.path.isfile(os.path.join(ROOT, m.group(1))), cmd


def test_summaries_are_short_text_with_their_commands():
    files = sorted(glob.glob(os.path.join(PROFILES, "*")))
    assert files
    for f in files:
        assert os.path.splitext(f)[1] in (".md", ".txt", ".json"), f
        assert os.path.getsize(f) < 16 * 1024, f
        if f.endswith(".json"):
            continue
        cmds = _commands(open(f).read())
        assert cmds, f"{f}: no command"
        for c in cmds:
            _check_command(c)


def test_traffic_record_names_known_workloads_and_classes():
    sys.path.insert(0, ROOT)
    import bench
    doc = json.load(open(os.path.join(PROFILES, "traffic.json")))
    for workload, policies in doc.items():
        assert workload in bench.WORKLOADS, workload
        for policy, classes in policies.items():
            assert policy in ("hybrid", "upper_bound", "learned"), policy
            for cls, ent in classes.items():
                assert cls in bench.KERNEL_SOURCES, cls
                assert ent["bytes_per_step"] > 0 and re.fullmatch(r"[0-9a-f]{16}", ent["source_digest"])
                _check_command(ent["command"])
