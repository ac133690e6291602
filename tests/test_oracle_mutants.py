"""Planted mistakes in the oracle must fail the pins.

Each mutant is a copy of oracle/slg_oracle.c with one plausible error
(a wrong comparison, a dropped term, a transposed operand, a missing reset),
compiled to a temporary library and run against the pin suite in a child
process (a broken oracle may crash).  The real oracle is not modified.
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "slg_oracle.c")

MUTANTS = {
    "self_loops": ("if (f <= e) continue;", "if (f < e) continue;"),
    "lower_triangle": ("if (f <= e) continue;", "if (f >= e) continue;"),
    "threshold_off_by_one": ("cnt[f] >= J->s", "cnt[f] > J->s"),
    "dropped_last_vertex": ("k < J->e_off[e + 1]; ++k) {\n    int32_t v",
                            "k < J->e_off[e + 1] - 1; ++k) {\n    int32_t v"),
    "no_reset": ("    cnt[f] = 0;\n", "\n"),
    "transposed_output": ("push(out, e, f, cnt[f])", "push(out, f, e, cnt[f])"),
    "unsorted_row": ("qsort(touched", "if (0) qsort(touched"),
    "double_count": ("if (cnt[f]++ == 0)", "cnt[f]++; if (cnt[f]++ == 0)"),
    "transpose_index": ("J->v_idx[fill[J->e_idx[k]]++] = e;",
                        "J->v_idx[fill[J->e_idx[k]]++] = e > 0 ? e - 1 : e;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new, 1))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC",
                           "-pthread", "-o", str(lib), str(mut)])
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})
        import pins
        fails = pins.run_all({str(lib)!r})
        print(len(fails)); print(fails[:3])
        sys.exit(0 if fails else 3)
    """)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True,
                       text=True, timeout=600)
    # exit 0: some pin failed (caught); non-zero other than 3: crashed (caught)
    assert r.returncode != 3, f"mutant {name} passed every pin:\n{r.stdout}"
