"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of the oracle's C source (on the CPU), builds it, and runs the
pin tests against the mutant: at least one pin has to fail."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gns_oracle.c")

MUTANTS = {
    "knuth_merge_takes_right_on_ties":
        ("if (ord_cmp(sk[j], sk[i], c->key_type, c->order) < 0) {",
         "if (ord_cmp(sk[j], sk[i], c->key_type, c->order) <= 0) {"),
    "frog_left_node_takes_left_on_ties":
        ("if (ord_cmp(f->k[j], f->k[i], kt, od) >= 0)", "if (ord_cmp(f->k[j], f->k[i], kt, od) > 0)"),
    "frog_right_node_takes_right_on_ties":
        ("if (ord_cmp(f->k[i], f->k[j], kt, od) <= 0)", "if (ord_cmp(f->k[i], f->k[j], kt, od) < 0)"),
    "negative_floats_not_reversed":
        ("return (ma < mb) ? 1 : -1;                 /* both negative: reversed */",
         "return (ma < mb) ? -1 : 1;"),
    "sign_order_flipped":
        ("if (sa != sb) return sa ? -1 : 1;", "if (sa != sb) return sa ? 1 : -1;"),
    "surplus_to_inner_side":
        ("n_outer = (p->n + 1) / 2;", "n_outer = p->n / 2;"),
    "outer_child_gets_extra_buffer":
        ("int64_t b_outer = n_outer / 2;", "int64_t b_outer = (n_outer + 1) / 2;"),
    "definition_ties_reversed":
        ("return (a->idx < b->idx) ? -1 : (a->idx > b->idx) ? 1 : 0;",
         "return (a->idx < b->idx) ? 1 : (a->idx > b->idx) ? -1 : 0;"),
    "descending_ignored":
        ("return order == ORC_DESC ? -c : c;", "return c;"),
    "int64_compared_unsigned":
        ("int64_t x = (int64_t)a, y = (int64_t)b;", "uint64_t x = a, y = b;"),
}

PINS = ["tests/test_oracle_bruteforce.py", "tests/test_oracle_frog.py",
        "tests/test_oracle_order.py", "tests/test_oracle_invariants.py"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not found: {name}"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mutant.c")
        so = os.path.join(td, "libmutant.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", c, "-o", so])
        env = dict(os.environ, GNS_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
