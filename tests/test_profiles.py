"""The committed ncu summaries that bench.py reads (per-element FP64
instruction counts and DRAM bytes) name the sources they were captured on
and carry their sha256; bench.py uses a summary only while those sources are
unchanged.  These checks run without a GPU: a summary that no longer matches
is reported as skipped (bench.py then reports the formula count and a null
traffic for that kernel), and its keys must parse."""
import hashlib
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_11133_gb300", "csrc")
SUMMARIES = ["k_assemble_lognormal_1m.txt", "k_assemble_dw_lognormal_1m.txt", "fp64_step_lognormal_1m.txt"]


def read_kv(name):
    kv = {}
    for line in open(os.path.join(ROOT, "profiles", name)):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    return kv


@pytest.mark.parametrize("name", SUMMARIES)
def test_summary_matches_its_sources(name):
    kv = read_kv(name)
    sources = kv["sources"].split()
    assert sources and all(os.path.exists(os.path.join(CSRC, s)) for s in sources)
    h = hashlib.sha256()
    for s in sources:
        with open(os.path.join(CSRC, s), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != kv["sources_sha256"]:
        pytest.skip(f"profiles/{name} was captured on other sources than the current {sources}")


def test_summary_figures_parse():
    asm = read_kv("k_assemble_lognormal_1m.txt")
    assert float(asm["fp64_inst_per_tet"]) > 0 and float(asm["dram_bytes_per_tet"]) > 0
    step = read_kv("fp64_step_lognormal_1m.txt")
    per = {k.split(" ", 1)[1]: float(v) for k, v in step.items() if k.startswith("fp64_per_tet ")}
    assert abs(sum(per.values()) - float(step["fp64_per_tet_total"])) < 1e-6
    assert per["k_assemble"] == float(asm["fp64_inst_per_tet"])
