"""The committed ncu summaries: every ncu command leaves the GPU clocks
alone (--clock-control none), each summary names the command that made it,
and the traffic notes the bench scales its roofline traffic from were taken
on the kernel sources as they are now (else the bench reports traffic as
null)."""
import glob
import hashlib
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))


def test_every_ncu_command_keeps_the_clocks():
    assert PROFILES
    for path in PROFILES:
        text = open(path).read()
        assert "python bench.py" in text, path
        cmds = [line for line in text.splitlines()
                if line.strip().startswith("ncu ")]
        for line in cmds:
            assert "--clock-control none" in line, (path, line)
        assert os.path.getsize(path) < 16 * 1024, path


def test_traffic_notes_match_the_kernel_sources():
    notes = [p for p in PROFILES if p.endswith("_traffic.txt")]
    assert notes
    for path in notes:
        text = open(path).read()
        src = re.search(r"kernel_source:\s*(\S+)", text).group(1)
        sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
        ratio = re.search(r"dram_bytes_per_\w+_byte:\s*([0-9.]+)", text)
        digest = hashlib.sha256(
            open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
        assert sha and sha.group(1) == digest, (path, src)
        assert ratio and 0.1 < float(ratio.group(1)) < 10.0
