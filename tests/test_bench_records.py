"""The committed profile records that bench.py reads, and the ncu commands
quoted in the profile summaries.

bench.py fills `roofline.traffic` and `roofline.issue` from per-launch
counter records under profiles/ (keyed by the dominant phase and workload);
a renamed phase or a lost record would silently drop those fields from the
bench line.  Every ncu command quoted in a summary must leave the GPU's
clocks alone (`--clock-control none`)."""
import glob
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_counter_records_have_the_bench_key():
    for name in ("traffic.json", "issue.json"):
        with open(os.path.join(PROFILES, name)) as f:
            rec = json.load(f)
        v = rec.get("bitset_count_rmat21_k4")
        assert isinstance(v, int) and v > 0, (name, v)
    # DRAM bytes per launch stay far below the algorithmic bytes of the
    # level 2 -> 3 rule on R-MAT 21 (41.8 GB: the graph is L2-resident), and
    # the instruction count is of the order the issue roof implies for a
    # ~20 ms launch (about 1.2e12 warp instructions/s at most)
    with open(os.path.join(PROFILES, "traffic.json")) as f:
        assert json.load(f)["bitset_count_rmat21_k4"] < 41.8e9
    with open(os.path.join(PROFILES, "issue.json")) as f:
        assert json.load(f)["bitset_count_rmat21_k4"] < 1.3e12 * 0.03


def test_profile_commands_leave_clocks_alone():
    for path in glob.glob(os.path.join(PROFILES, "*.md")):
        with open(path) as f:
            text = f.read()
        # a quoted command sits in a fenced block, starts with `ncu ` at the
        # start of a line and goes on over the lines that end with a backslash
        lines = text.split("\n")
        fenced = False
        for i, line in enumerate(lines):
            if line.lstrip().startswith("```"):
                fenced = not fenced
                continue
            if not fenced or not re.match(r"\s*ncu\s", line):
                continue
            cmd = [line]
            while cmd[-1].rstrip().endswith("\\") and i + len(cmd) < len(lines):
                cmd.append(lines[i + len(cmd)])
            cmd = " ".join(cmd)
            assert "--clock-control none" in cmd, (os.path.basename(path), cmd[:120])
