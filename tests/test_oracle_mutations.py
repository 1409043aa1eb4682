"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of the oracle's source (on the CPU): the C oracle is built
from the copy, the learned path's Python oracle is loaded from it, and the pin
tests run against the mutant: at least one pin has to fail."""
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
    # adaptive sorts (Full adaptivity, Symmetric merging and Squidsort sections)
    "omit_half_in_buffer_not_brought_back":
        ("if (a.reg != b.reg) {                 /* bring the half", "if (0) {                 /* bring the half"),
    "omit_non_overlap_test_dropped":
        ("if (oL == ORI_ASC ? c <= 0 : c > 0) {", "if (0) {"),
    "octo_mirrored_run_omits_on_equal_keys":
        ("if (oL == ORI_ASC ? c <= 0 : c > 0) {", "if (oL == ORI_ASC ? c <= 0 : c >= 0) {"),
    "octo_pair_of_equal_keys_mirrored":
        ("res.ori = ord_cmp(k[m], k[m - 1], kt, od) < 0 ? ORI_DESC : ORI_ASC;",
         "res.ori = ord_cmp(k[m], k[m - 1], kt, od) <= 0 ? ORI_DESC : ORI_ASC;"),
    "gecko_orientation_sides_swapped":
        ("const int o = x->side == 0 ? ORI_ASC : ORI_DESC;", "const int o = x->side == 0 ? ORI_DESC : ORI_ASC;"),
    "symmetric_largest_first_takes_left_on_ties":
        ("(lf ? ord_cmp(f->k[a], f->k[b], kt, od) > 0 :", "(lf ? ord_cmp(f->k[a], f->k[b], kt, od) >= 0 :"),
    "squid_non_overlap_test_dropped":
        ("sym_merge(s, x, &L, oL, &R, oR, o, 1);", "sym_merge(s, x, &L, oL, &R, oR, o, 0);"),
}

PINS = ["tests/test_oracle_bruteforce.py", "tests/test_oracle_frog.py",
        "tests/test_oracle_order.py", "tests/test_oracle_invariants.py", "tests/test_oracle_adaptive.py"]


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


MLP_SRC = os.path.join(ROOT, "oracle", "mlp.py")

MLP_MUTANTS = {
    "bucket_counts_splitters_below_only": ('side="right"', 'side="left"'),
    "output_tanh_derivative_dropped": ("dz3 = dy * (1.0 - y * y)", "dz3 = dy"),
    "w2_transposed_in_forward_and_gradient": ("h2 = np.tanh(h1 @ w2.T + b2)", "h2 = np.tanh(h1 @ w2 + b2)"),
    "adam_first_moment_not_bias_corrected": ("mh = m1 / (1 - beta1 ** step)", "mh = m1"),
    "adam_second_moment_not_bias_corrected": ("vh = m2 / (1 - beta2 ** step)", "vh = m2"),
    "layer1_gradient_sign_flipped": ("g_w1 = dz1.T @ x", "g_w1 = -(dz1.T @ x)"),
}


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_mlp_pins_catch_mutant(name):
    old, new = MLP_MUTANTS[name]
    src = open(MLP_SRC).read()
    assert src.count(old) == 1, f"mutation site not found: {name}"
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "mlp_mutant.py")
        open(path, "w").write(src.replace(old, new))
        env = dict(os.environ, GNS_ORACLE_MLP=path)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "tests/test_oracle_mlp.py"], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
