"""The ctypes binding mirrors include/ttc.h by hand: its structures, the
status codes and the tuners' candidate tables.  These CPU tests compile a
small C program against the header with the host compiler and check that
every structure the binding passes across the C ABI has the header's size,
field order, field offsets and field sizes, and that the constants agree."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2106_02762_gb300 import ttc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttc.h")

# C structure name -> the binding's ctypes mirror
STRUCTS = {
    "ttc_delta": ttc.Delta,
    "ttc_load_opts": ttc.LoadOpts,
    "ttc_graph_stats": ttc.GraphStats,
    "ttc_kernel_time": ttc.KernelTime,
    "ttc_server_opts": ttc.ServerOpts,
    "ttc_server_stats": ttc.ServerStats,
}


def header_text():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def header_struct_fields(name):
    """Field names of `typedef struct { ... } name;`, in declaration order."""
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", header_text())
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "type a, b[4], c": drop the type words before the first declarator
        parts = [p.strip() for p in decl.split(",")]
        first = parts[0].split()[-1]
        for p in [first] + parts[1:]:
            fields.append(re.sub(r"\[.*\]", "", p).lstrip("*"))
    return fields


def header_constants():
    """Every integer constant the header defines: macros and ttc_status."""
    text = header_text()
    names = re.findall(r"^#define[ \t]+(TTC_[A-Z0-9_]+)[ \t]+\S", text, flags=re.M)
    m = re.search(r"typedef\s+enum\s*\{([^{}]*)\}\s*ttc_status\s*;", text)
    assert m
    names += re.findall(r"\b(TTC_[A-Z0-9_]+)\s*=", m.group(1))
    return names


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ttc.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s *)0)->%s));'
                         % (cname, f, cname, f, cname, f))
    lines.append('  for (int i = 0; i < TTC_TUNE_CANDIDATES; i++) printf("light %u\\n", ttc_tune_candidates[i]);')
    lines.append('  for (int i = 0; i < TTC_TUNE_HEAVY_CANDIDATES; i++) printf("heavy %u %u %u\\n", '
                 'ttc_tune_heavy_candidates[i][0], ttc_tune_heavy_candidates[i][1], ttc_tune_heavy_candidates[i][2]);')
    for name in header_constants():
        lines.append('  printf("const %s %%lld\\n", (long long)%s);' % (name, name))
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [ln.split() for ln in out.splitlines()]


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_field_order_matches_header(cname):
    assert [f for f, _ in STRUCTS[cname]._fields_] == header_struct_fields(cname)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(probe, cname):
    import ctypes
    cls = STRUCTS[cname]
    rows = {r[1]: r[2:] for r in probe if r[0] == cname}
    assert int(rows.pop("sizeof")[0]) == ctypes.sizeof(cls)
    for f, _ in cls._fields_:
        off, size = map(int, rows[f])
        desc = getattr(cls, f)
        assert (desc.offset, desc.size) == (off, size), (cname, f)


def test_tuner_candidates_match_header(probe):
    light = tuple(int(r[1]) for r in probe if r[0] == "light")
    heavy = tuple((int(r[1]), int(r[2]), int(r[3])) for r in probe if r[0] == "heavy")
    assert light == ttc.TUNE_CANDIDATES
    assert heavy == ttc.TUNE_HEAVY_CANDIDATES


def test_constants_match_header(probe):
    consts = {r[1]: int(r[2]) for r in probe if r[0] == "const"}
    status = {k: v for k, v in consts.items() if k.startswith("TTC_ERR_")}
    assert len(status) == 9 and len(ttc.STATUS) == 9
    for name, code in status.items():
        assert ttc.STATUS[code] == name[len("TTC_ERR_"):], name
    assert (consts["TTC_OK"], consts["TTC_PENDING"]) == (ttc.OK, ttc.PENDING)
    mirrored = [k for k in consts if k.startswith(("TTC_LOAD_", "TTC_ORIENT_", "TTC_LABEL_", "TTC_HEAVY_"))]
    assert len(mirrored) == 12
    for name in mirrored + ["TTC_NUM_TYPES"]:
        assert getattr(ttc, name[len("TTC_"):]) == consts[name], name
    assert consts["TTC_TUNE_CANDIDATES"] == len(ttc.TUNE_CANDIDATES)
    assert consts["TTC_TUNE_HEAVY_CANDIDATES"] == len(ttc.TUNE_HEAVY_CANDIDATES)
