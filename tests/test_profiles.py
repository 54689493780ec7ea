"""The committed ncu summaries: every one names the command that made it (committed files only,
clocks left alone), and the traffic table the bench line reads points at them."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def test_traffic_table_entries():
    with open(os.path.join(PROF, "traffic.json")) as fh:
        d = json.load(fh)
    assert "k_window_mixed_NT128_N67108864" in d   # the bench line's dominant kernel
    for key, ent in d.items():
        assert ent["dram_bytes_per_launch"] == ent["dram_bytes_read"] + ent["dram_bytes_write"] > 0, key
        assert re.fullmatch(r"[0-9a-f]{16}", ent["src_hash"]), key
        assert os.path.exists(os.path.join(ROOT, ent["summary"])), key


def test_summaries_name_their_commands():
    mds = [f for f in os.listdir(PROF) if f.endswith(".md")]
    assert mds
    for f in mds:
        with open(os.path.join(PROF, f)) as fh:
            text = fh.read()
        cmds = re.findall(r"```\n(.*?)```", text, re.S)
        assert cmds, f
        for block in cmds:
            for line in block.strip().splitlines():
                if line.startswith("ncu"):
                    assert "--clock-control none" in line, (f, line)
                assert "_work" not in line and "/root" not in line, (f, line)
                assert "bench.py" in line, (f, line)
