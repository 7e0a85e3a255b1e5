"""The ncu summaries under profiles/ against what the benchmark reports.

bench.py reports, beside each product kernel's roofline, the DRAM traffic per
launch that an ncu capture measured, keyed by a hash of the kernel sources
and naming the summary it came from.  These checks keep the two in step: the
named summary exists, states the same read + write traffic, and every ncu
command in profiles/ leaves the GPU clocks alone.
"""
import os
import re

import bench

PROFILES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")


def test_traffic_table_matches_the_named_summaries():
    assert bench.NCU_TRAFFIC, "no captured traffic"
    for (kernel, workload), (traffic, src_hash, path) in bench.NCU_TRAFFIC.items():
        full = os.path.join(os.path.dirname(PROFILES), path)
        assert os.path.exists(full), path
        text = open(full).read()
        assert kernel in text.splitlines()[0], f"{path} does not cover {kernel}"
        m = re.search(r"\| traffic \(read \+ write\) \| ([0-9.]+) MB \|", text)
        assert m, f"{path} states no read + write traffic"
        assert abs(float(m.group(1)) * 1e6 - traffic) <= 0.05e6, (path, m.group(1), traffic)
        assert re.fullmatch(r"[0-9a-f]{16}", src_hash)


def test_all_entries_belong_to_one_build():
    # the table is refreshed as a whole after a capture of the current sources
    assert len({h for _, h, _ in bench.NCU_TRAFFIC.values()}) == 1


def test_every_ncu_command_keeps_the_clocks():
    for name in sorted(os.listdir(PROFILES)):
        text = open(os.path.join(PROFILES, name)).read()
        for line in text.splitlines():
            if re.match(r"\s*ncu\s+-", line):  # a command line, not prose
                assert "--clock-control none" in line, f"{name}: {line.strip()}"
