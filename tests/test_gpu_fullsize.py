"""Full-size checks at the benchmark's workload (2^27 float64 keys + uint32
index payload, four patterns, both tiers), in the benchmark's launch
configuration: invariants that hold at any size plus sampled output positions
computed one by one by the oracle."""
import numpy as np
import pytest

import oracle
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu

N_FULL = 1 << 27


def check_sorted_stable(keys_in, k_out, p_out, order=0, samples=12, seed=0):
    n = keys_in.size
    # a permutation carried by the payload, moving the original bit patterns
    assert np.array_equal(np.sort(p_out), np.arange(n, dtype=np.uint32))
    assert np.array_equal(k_out.view(np.uint64), keys_in.view(np.uint64)[p_out])
    # finite keys without -0.0: order by float comparison; ties in input order
    d = np.diff(k_out)
    if order == 0:
        assert np.all(d >= 0)
    else:
        assert np.all(d <= 0)
    eq = d == 0
    assert np.all(p_out[1:][eq] > p_out[:-1][eq])
    # sampled final positions from the oracle (rank counting, one by one)
    rng = np.random.default_rng(seed)
    for i in rng.integers(0, n, samples):
        pos = oracle.final_position(keys_in, int(i), oracle.DESC if order else oracle.ASC)
        assert p_out[pos] == i


@pytest.mark.parametrize("bf", [1.0, 0.5])
@pytest.mark.parametrize("pattern", inputs.PATTERNS_C1)
def test_config_full_size(pattern, bf):
    need_gpu()
    import paper_2402_01816_gb300 as g
    keys = inputs.make_keys(pattern, N_FULL, seed=0)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(N_FULL))
    g.gns_sort(kt, pt, buffer_fraction=bf)
    assert g.gns_stream_status() == 0
    k_out = kt.cpu().numpy()
    p_out = pt.cpu().numpy().view(np.uint32)
    del kt, pt
    torch.cuda.empty_cache()
    check_sorted_stable(keys, k_out, p_out)


@pytest.mark.parametrize("variant", ["gecko", "squid"])
@pytest.mark.parametrize("pattern", ["permut", "desc_ties", "desc_runs"])
def test_symmetric_full_size(pattern, variant):
    """gns_sort_symmetric at the benchmark's size (2^27 keys, 50% buffer), on
    random input and on the inputs whose runs the variants store mirrored:
    invariants plus sampled positions from the oracle."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    keys = inputs.make_keys(pattern, N_FULL, seed=0)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(N_FULL))
    g.gns_sort_symmetric(kt, pt, variant=g.GECKOSORT1 if variant == "gecko" else g.SQUIDSORT1)
    assert g.gns_stream_status() == 0
    k_out = kt.cpu().numpy()
    p_out = pt.cpu().numpy().view(np.uint32)
    del kt, pt
    torch.cuda.empty_cache()
    check_sorted_stable(keys, k_out, p_out, seed=1)


def test_small_config_exact():
    """2^20 uniform[0,1) keys, ascending, 100% buffer: bit-exact against the
    oracle's full stable sort."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = 1 << 20
    keys = inputs.make_keys("uniform", n, seed=0)
    pay = inputs.index_payload(n)
    kt, pt = to_dev_keys(keys), to_dev_payload(pay)
    g.gns_sort(kt, pt, buffer_fraction=1.0)
    want_k, want_p = oracle.stable_sort(keys, pay)
    assert np.array_equal(kt.cpu().numpy().view(np.uint64), want_k.view(np.uint64))
    assert np.array_equal(pt.cpu().numpy().view(np.uint32), want_p)


N_LARGE = 1 << 31


@pytest.mark.parametrize("learned", [False, True])
@pytest.mark.parametrize("pattern", ["permut", "presorted_runs"])
def test_large_low_memory_run(pattern, learned):
    """2^31 float64 keys + uint32 index payload at the 50% buffer tier (24 GiB
    of data, 12 GiB of buffer), by the plain and by the learned-splitter sort.
    Both patterns are permutations of 1..n, so the sorted keys must be exactly
    1..n and the payload must carry every key from its input position; checked
    on the device."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    kt = inputs.make_keys_device(pattern, N_LARGE, seed=0)
    pt = torch.arange(N_LARGE, dtype=torch.int64, device="cuda").to(torch.int32)
    k_in = kt.clone()
    kind = 1 if learned else 0
    assert 1.0 + g.gns_workspace_bytes(N_LARGE, 0.5, kind) / (12.0 * N_LARGE) < 1.52     # %RAM
    if learned:
        rep = g.gns_learned_sort(kt, pt, buffer_fraction=0.5, report=True)
        assert rep["fallback"] == 0
    else:
        g.gns_sort(kt, pt, buffer_fraction=0.5)
    assert g.gns_stream_status() == 0
    want = torch.arange(1, N_LARGE + 1, dtype=torch.float64, device="cuda")
    assert torch.equal(kt, want)
    del want
    idx = pt.to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(k_in[idx], kt)
    del k_in, kt, pt, idx
    torch.cuda.empty_cache()
