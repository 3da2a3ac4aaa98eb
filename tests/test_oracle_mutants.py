"""The pins catch plausible oracle mistakes.  Each case plants one mistake
in a copy of oracle/ttc_oracle.c (a window bound off by one, a swapped type,
a reversed tie-break, a dropped term of Lemma 1, a missing role assignment),
compiles it, and checks that at least one paper-derived pin (Table 1 cells,
the hand-worked Def. 1 / Fig. 2 cases, the unbounded-window product) fails.
The mistakes are planted on the CPU only."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2106_02762_gb300 import synth
from tests.golden import readers

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "ttc_oracle.c")
BIG = 1 << 40

MUTANTS = {
    "d12_strict_in_bruteforce_and_lemma1": [
        ("(i128)e2->t - e1->t <= d12", "(i128)e2->t - e1->t < d12"),
        ("if (gap12 > d12) continue;", "if (gap12 >= d12) continue;"),
    ],
    "types_T1_T2_swapped": [
        ("if (e2_cb && e3_ac) return 0;\n    if (e2_cb && e3_ca) return 1;",
         "if (e2_cb && e3_ac) return 1;\n    if (e2_cb && e3_ca) return 0;"),
    ],
    "types_T6_T8_swapped": [
        ("if (e2_ca && e3_cb) return 5;", "if (e2_ca && e3_cb) return 7;"),
        ("if (e2_ca && e3_bc) return 7;", "if (e2_ca && e3_bc) return 5;"),
    ],
    "tie_break_reversed": [
        ("a->t < b->t || (a->t == b->t && a->idx < b->idx)", "a->t < b->t || (a->t == b->t && a->idx > b->idx)"),
    ],
    "lemma1_min_dropped": [
        ("if ((i128)e1->t + d13 < bound) bound = (i128)e1->t + d13;", ""),
        ("&& (i128)e3->t - e1->t <= d13", ""),
    ],
    "third_window_strict": [
        ("if ((i128)s->e[mid]->t <= bound) l = mid + 1;", "if ((i128)s->e[mid]->t < bound) l = mid + 1;"),
        ("(i128)e3->t - e2->t <= d23", "(i128)e3->t - e2->t < d23"),
    ],
    "one_role_assignment_missing": [
        ("for (int r = 0; r < 6; r++) lemma1_roles", "for (int r = 0; r < 5; r++) lemma1_roles"),
    ],
}


def _build(name, edits, tmp):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, (name, old)
        src = src.replace(old, new)
    c = tmp / (name + ".c")
    c.write_text(src)
    so = tmp / (name + ".so")
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    p, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    lib.ttc_oracle_bruteforce.argtypes = [p, p, p, u64, p, u32, p]
    lib.ttc_oracle_count.argtypes = [p, p, p, u64, p, u32, i32, p]
    return lib


def _run(fn, s, d, t, deltas, *extra):
    s = np.ascontiguousarray(s, np.uint32)
    d = np.ascontiguousarray(d, np.uint32)
    t = np.ascontiguousarray(t, np.int64)
    q = np.ascontiguousarray(np.asarray(deltas, np.int64).reshape(-1, 3))
    out = np.zeros((q.shape[0], 8), np.uint64)
    fn(s.ctypes.data, d.ctypes.data, t.ctypes.data, s.size, q.ctypes.data, q.shape[0], *extra, out.ctypes.data)
    return out


def _pins_hold(lib):
    """True when every pin passes for this build."""
    evals = [lambda *a: _run(lib.ttc_oracle_bruteforce, *a), lambda *a: _run(lib.ttc_oracle_count, *a, 1)]
    orders, orients, psi = readers.psi_table()
    for k in range(1, 7):
        for r in range(1, 9):
            name = dict(zip("uvw", (0, 1, 2)))
            t_of = {frozenset(pp): i + 1 for i, pp in enumerate(orders[k])}
            e = np.asarray([(name[x[0]], name[x[1]], t_of[frozenset(x)]) for x in orients[r]], np.int64)
            exp = np.zeros(8, np.uint64)
            exp[psi[k][r] - 1] = 1
            for ev in evals:
                if not (ev(e[:, 0], e[:, 1], e[:, 2], [(BIG, BIG, BIG)])[0] == exp).all():
                    return False
    for _, edges, checks in readers.hand_cases():
        e = np.asarray(edges, np.int64)
        exp = np.asarray([c[1] for c in checks], np.uint64)
        for ev in evals:
            if not (ev(e[:, 0], e[:, 1], e[:, 2], [c[0] for c in checks]) == exp).all():
                return False
    for seed in range(10):
        s, d, t = synth.random_tiny(3000 + seed, 6, 30, 4)
        key = {}
        for a, b in zip(s.tolist(), d.tolist()):
            if a != b:
                key[frozenset((a, b))] = key.get(frozenset((a, b)), 0) + 1
        verts = sorted({v for p in key for v in p})
        prod = 0
        for i, a in enumerate(verts):
            for j, b in enumerate(verts[i + 1:], i + 1):
                for c in verts[j + 1:]:
                    ab, ac, bc = frozenset((a, b)), frozenset((a, c)), frozenset((b, c))
                    if ab in key and ac in key and bc in key:
                        prod += key[ab] * key[ac] * key[bc]
        for ev in evals:
            if int(ev(s, d, t, [(BIG, BIG, BIG)]).sum()) != prod:
                return False
    return True


def test_unmutated_oracle_passes_the_pins(tmp_path):
    assert _pins_hold(_build("original", [], tmp_path))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    assert not _pins_hold(_build(name, MUTANTS[name], tmp_path)), name
