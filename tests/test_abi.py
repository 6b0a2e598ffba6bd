"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/sr.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "sr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sr_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    from paper_1805_00106_gb300 import sr
    path = sr._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(sr_\w+)", out))
    names = declared()
    assert len(names) >= 30
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = sr.lib()
    for n in names:
        assert hasattr(L, n)


def test_calls_fail_loudly_without_gpu():
    import torch
    from paper_1805_00106_gb300 import sr
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sr.SrError) as e:
        sr.Session.open([b"ACGT" * 64])
    assert e.value.status == sr.SR_ECUDA
    with pytest.raises(sr.SrError):
        sr.probe_dpx()


def test_binding_has_no_compute_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1805_00106_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cpp", ".cu", ".h")):
                src = open(os.path.join(dp, f), errors="replace").read()
                assert "oracle" not in src.replace("the oracle", ""), f


def test_tune_table_roundtrip(tmp_path):
    from paper_1805_00106_gb300 import sr
    bins = sr.tune_get()
    assert len(bins) >= 8 and bins[-1][0] == 256
    assert all(b[1] * b[2] >= b[0] for b in bins)
    p = str(tmp_path / "tune.txt")
    sr.lib().sr_tune_save(p.encode())
    # another valid table: every bin on a 32-lane shape that covers it
    new = [(b[0], 32, max(4, -(-b[0] // 32))) for b in bins]
    new = [(u, g, r if r in (4, 5, 6, 7, 8) else 8) for u, g, r in new]
    sr.tune_set(new)
    assert sr.tune_get() == new
    assert sr.lib().sr_tune_load(p.encode()) == 0
    assert sr.tune_get() == bins
    with pytest.raises(sr.SrError):
        sr.tune_set([(64, 4, 8)] + bins[1:])  # rows do not cover the bin


# each ctypes structure of the binding and the C type it mirrors
LAYOUTS = {"IndexParams": "sr_index_params", "Reads": "sr_reads", "CandParams": "sr_cand_params",
           "CandList": "sr_cand_list", "ScoreParams": "sr_score_params", "AlignOpts": "sr_align_opts",
           "Hit": "sr_hit", "Results": "sr_results", "ReportHit": "sr_report_hit", "Report": "sr_report",
           "SamOpts": "sr_sam_opts"}


def test_binding_structs_match_the_header(tmp_path):
    """Every structure the binding passes across the C ABI has the size and the
    field offsets of its declaration in include/sr.h, as gcc lays it out."""
    import ctypes

    from paper_1805_00106_gb300 import sr
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sr.h"', "int main(void) {"]
    for py, c in LAYOUTS.items():
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for f, _ in getattr(sr, py)._fields_:
            lines.append(f'  printf("{py} {f} %zu\\n", offsetof({c}, {f}));')
    lines.append("  return 0;\n}")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) == sum(1 + len(getattr(sr, py)._fields_) for py in LAYOUTS)
    for line in out:
        py, what, val = line.split()
        cls = getattr(sr, py)
        expect = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert int(val) == expect, (py, what, int(val), expect)


# binding constant -> the header's name for it
CONSTANTS = {"SR_OK": "SR_OK", "SR_EINVAL": "SR_EINVAL", "SR_ENOMEM": "SR_ENOMEM", "SR_ECUDA": "SR_ECUDA",
             "SR_EBADBASE": "SR_EBADBASE", "SR_ETIMEOUT": "SR_ETIMEOUT", "SR_EBUSY": "SR_EBUSY",
             "SR_EIO": "SR_EIO", "MODE_LOCAL": "SR_MODE_LOCAL", "MODE_FINAL_ROW": "SR_MODE_FINAL_ROW",
             "ENGINE_BATCHED": "SR_ENGINE_BATCHED", "ENGINE_PLAIN": "SR_ENGINE_PLAIN",
             "CLASS_UNALIGNED": "SR_CLASS_UNALIGNED", "CLASS_A": "SR_CLASS_A", "CLASS_B": "SR_CLASS_B",
             "CLASS_AMBIGUOUS": "SR_CLASS_AMBIGUOUS", "CIGAR_STRIDE": "SR_CIGAR_STRIDE",
             "REPORT_BEST_N": "SR_REPORT_BEST_N", "REPORT_TIED": "SR_REPORT_TIED", "REPORT_MAX": "SR_REPORT_MAX",
             "FLAG_DEVICE": "SR_FLAG_DEVICE"}


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, modes, engines, classes and limits the binding names have
    the header's values."""
    from paper_1805_00106_gb300 import sr
    body = "\n".join(f'  printf("{py} %lld\\n", (long long)({c}));' for py, c in CONSTANTS.items())
    src, exe = tmp_path / "consts.c", tmp_path / "consts"
    src.write_text('#include <stdio.h>\n#include "sr.h"\nint main(void) {\n' + body + "\n  return 0;\n}\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) == len(CONSTANTS)
    for line in out:
        py, val = line.split()
        assert getattr(sr, py) == int(val), (py, getattr(sr, py), int(val))
