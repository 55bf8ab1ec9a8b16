"""The committed ncu records describe the committed code: every DRAM traffic
record in profiles/dram_traffic.json is keyed by a kernel role and workload
that the bench reports, was taken with the bench's committed launch plan
for that workload, and lists kernel sources whose hashes match the files
(so the bench reports the traffic rather than null); each workload has a
summary with the full command."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_records_match_plans_and_sources():
    d = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    assert d["kernels"]
    for key, rec in d["kernels"].items():
        role, workload = key.split("@")
        assert role in ("sweep_x_h1", "sweep_y", "sweep_z"), key
        assert rec["plan"] == bench.PLANS[workload], (key, rec["plan"])
        for name, sha in rec["sources"].items():
            path = os.path.join(ROOT, "paper_1906_06327_gb300", "csrc", name)
            assert hashlib.sha256(open(path, "rb").read()).hexdigest() == sha, (key, name)
        assert bench._traffic(role, workload, rec["plan"]) == rec["dram_bytes_per_launch"]
        # DRAM bytes of one sweep: at most the algorithmic read + write of the
        # state plus 15% (re-reads), at least a third of it (L2 hits)
        sites = 1
        for v in bench._workload(workload).n:
            sites *= v
        algo = 16 * sites
        assert algo / 3 <= rec["dram_bytes_per_launch"] <= 1.15 * algo, (key, rec)


def test_every_profiled_workload_has_a_summary_with_its_command():
    d = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    for workload in {k.split("@")[1] for k in d["kernels"]}:
        text = open(os.path.join(ROOT, "profiles", f"sweeps_{workload}.md")).read()
        assert "ncu " in text and "--clock-control none" in text
        assert bench.PLANS[workload] in text
