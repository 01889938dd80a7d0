"""The committed ncu summaries: text only, each with the command that made
it, and every recorded DRAM-traffic figure in the form the benchmark reads
(so a figure taken on other device code is ignored, not misread)."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
TRAFFIC = re.compile(r"traffic:\s*kernel=(\S+)\s+workload=(\S+)\s+bytes_per_launch=(\d+)"
                     r"(?:\s+passes=(\d+))?\s+sources=(\w+)")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_for_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _summaries():
    return sorted(f for f in os.listdir(PROFILES) if not f.startswith("."))


def test_summaries_are_short_text_with_their_command():
    names = _summaries()
    assert names
    for name in names:
        assert name.endswith((".md", ".txt")), name
        path = os.path.join(PROFILES, name)
        assert os.path.getsize(path) < 16 * 1024, name
        text = open(path).read()
        assert "ncu " in text and "--clock-control none" in text, name


def test_traffic_records_parse_and_are_plausible():
    found = 0
    for name in _summaries():
        for m in TRAFFIC.finditer(open(os.path.join(PROFILES, name)).read()):
            found += 1
            kernel, workload, nbytes, passes, sources = m.groups()
            assert re.fullmatch(r"[0-9a-f]{16}", sources), (name, sources)
            # one pass over 2^28 int32 keys moves 2 x 4 B x 2^28 algorithmic
            # bytes (a persistent merge launch runs `passes` of them); DRAM
            # traffic within 10% of that (writes may stay in L2)
            if workload.startswith("int32_2e28"):
                per_pass = int(nbytes) / int(passes or 1)
                assert 0.9 * 2 * 4 * 2**28 <= per_pass <= 1.1 * 2 * 4 * 2**28, (name, nbytes, passes)
    assert found >= 1


def test_benchmark_reads_a_record_only_for_matching_device_code():
    bench = _bench()
    digest = bench.kernel_digest()
    recs = [m.groups() for name in _summaries()
            for m in TRAFFIC.finditer(open(os.path.join(PROFILES, name)).read())]
    recs = [(k, w, b, src) for k, w, b, _, src in recs]
    for kernel, workload, nbytes, sources in recs:
        got = bench.traffic_from_profiles(kernel, workload)
        if sources == digest:
            assert got == int(nbytes)
        else:
            assert got is None or any(r[0] == kernel and r[1] == workload and r[3] == digest for r in recs)


INSTR = re.compile(r"instructions:\s*kernel=(\S+)\s+thread_instructions_per_key=([0-9.]+)\s+sources=(\w+)")


def test_instruction_records_parse_and_are_read_only_for_matching_code():
    bench = _bench()
    digest = bench.kernel_digest()
    for name in _summaries():
        for m in INSTR.finditer(open(os.path.join(PROFILES, name)).read()):
            kernel, ipk, sources = m.groups()
            assert re.fullmatch(r"[0-9a-f]{16}", sources), (name, sources)
            assert 10.0 < float(ipk) < 1000.0, (name, ipk)
            got = bench.instructions_from_profiles(kernel)
            if sources == digest:
                assert got == float(ipk)
