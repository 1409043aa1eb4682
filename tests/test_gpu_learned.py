"""The learned-splitter sort and its network's kernels.

* forward, loss and gradient of the network match the float64 oracle
  (oracle/mlp.py, itself pinned by finite differences) within float32 error;
* one Adam step of the on-device trainer matches the oracle's Adam step;
* training reduces the loss;
* the learned sort is bit-exact against the oracle's stable sort (it must be,
  whatever the network learned), including ties, NaNs, signed zeros, both
  orders, keys only, and its fallbacks;
* the trained network balances the buckets far better than evenly spaced
  splitters (what the network gains over the method without it);
* the half-buffer form (buffer_fraction in [0.5, 1)) is bit-exact too;
* the full learned workload: 2^28 float64 keys from the three-part mixture.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2402_01816_gb300 import inputs
from tests.gpu_util import assert_bitexact, need_gpu, to_dev_keys, to_dev_payload, torch

pytestmark = pytest.mark.gpu


def _rand_params(seed):
    rng = np.random.default_rng(seed)
    import paper_2402_01816_gb300 as g
    p = g.gns_mlp_init_params().astype(np.float64)
    p += rng.normal(0, 0.05, p.size)
    return p.astype(np.float32)


def test_forward_matches_oracle():
    need_gpu()
    import paper_2402_01816_gb300 as g
    p = _rand_params(1)
    x = np.random.default_rng(2).random(5000).astype(np.float32)
    y = g.gns_mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(y - want)) < 2e-5


def test_loss_and_gradient_match_oracle():
    need_gpu()
    import paper_2402_01816_gb300 as g
    p = _rand_params(3)
    rng = np.random.default_rng(4)
    x = rng.random(4096).astype(np.float32)
    t = np.sort(rng.random(4096)).astype(np.float32)
    loss, grad = g.gns_mlp_loss_grad(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda(),
                                     torch.from_numpy(t).cuda())
    wl, wg = mlp.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - wl) <= 1e-4 * abs(wl) + 1e-7
    grad = grad.cpu().numpy()
    scale = np.max(np.abs(wg))
    assert np.max(np.abs(grad - wg)) <= 2e-3 * scale
    # every block of the parameter vector, not just the largest entries
    for a, b in [(mlp.W1, mlp.B1), (mlp.B1, mlp.W2), (mlp.W2, mlp.B2), (mlp.B2, mlp.W3), (mlp.W3, mlp.B3)]:
        s = np.max(np.abs(wg[a:b])) + 1e-12
        assert np.max(np.abs(grad[a:b] - wg[a:b])) <= 5e-3 * s, (a, b)


def test_one_adam_step_matches_oracle():
    need_gpu()
    import paper_2402_01816_gb300 as g
    m, batch = 1 << 12, 1024
    p = _rand_params(5)
    rng = np.random.default_rng(6)
    x = np.sort(rng.random(m)).astype(np.float32)
    t = ((np.arange(m) + 0.5) / m).astype(np.float32)
    out, loss = g.gns_mlp_train(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(p).cuda(),
                                steps=1, batch=batch, learning_rate=1e-2)
    idx = (np.arange(batch, dtype=np.uint64) * np.uint64(40503)) & np.uint64(m - 1)
    wl, wg = mlp.loss_grad(p.astype(np.float64), x[idx].astype(np.float64), t[idx].astype(np.float64))
    want, _, _ = mlp.adam_step(p.astype(np.float64), wg, np.zeros(p.size), np.zeros(p.size), 1, lr=1e-2)
    got = out.cpu().numpy()
    # the first Adam step moves every parameter by about lr * sign(g); entries with
    # a tiny gradient may flip sign in float32, so compare where |g| is not tiny
    big = np.abs(wg) > 1e-3 * np.max(np.abs(wg))
    assert np.max(np.abs(got[big] - want[big])) < 1e-4
    assert abs(loss.item() - wl) <= 1e-3 * abs(wl) + 1e-7


def _key53(keys):
    """53-bit prefixes of order-mapped float64 keys (input preparation only)."""
    b = keys.view(np.uint64)
    enc = np.where(b >> np.uint64(63), ~b, b | np.uint64(1 << 63))
    return enc >> np.uint64(11)


def test_training_reduces_loss():
    """The trainer fits a wavy correction (four periods of a sine) with the
    same kernels the sort uses."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    m = 1 << 16
    x = ((np.arange(m) + 0.5) / m).astype(np.float32)
    t = (0.5 * np.sin(8 * np.pi * x)).astype(np.float32)
    p0 = torch.from_numpy(g.gns_mlp_init_params()).cuda()
    xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0, _ = g.gns_mlp_loss_grad(p0, xt, tt)
    p1, _ = g.gns_mlp_train(xt, tt, p0, steps=256)
    l1, _ = g.gns_mlp_loss_grad(p1, xt, tt)
    assert abs(l0.item() - 0.125) < 1e-3                      # initial correction is zero
    assert l1.item() < 0.1 * l0.item(), (l0.item(), l1.item())


def _learned(keys, order=0, with_payload=True, **kw):
    import paper_2402_01816_gb300 as g
    n = keys.size
    pay = inputs.index_payload(n)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(pay) if with_payload else None
    rep = g.gns_learned_sort(kt, pt, order=order, report=True, **kw)
    assert g.gns_stream_status() == 0
    want_k, want_p = oracle.stable_sort(keys, pay if with_payload else None, oracle.DESC if order else oracle.ASC)
    got_p = None if pt is None else pt.cpu().numpy().view(np.uint32)
    assert_bitexact(kt.cpu().numpy(), got_p, want_k, want_p)
    return rep


N = (1 << 20) + 4099


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("pattern", ["mixture", "uniform", "ties", "permut", "asc_noise", "desc"])
def test_learned_exact(pattern, order):
    need_gpu()
    rep = _learned(inputs.make_keys(pattern, N, seed=11), order=order)
    assert rep["fallback"] == 0 and rep["nonempty_buckets"] >= 1


def test_learned_edge_keys_and_keys_only():
    need_gpu()
    alpha = inputs.edge_alphabet()
    rng = np.random.default_rng(12)
    keys = np.concatenate([alpha[rng.integers(0, alpha.size, N // 2)], rng.normal(size=N - N // 2)])
    _learned(keys, order=0)
    _learned(keys, order=1, with_payload=False)
    _learned(np.full(N, 3.0))                                 # all equal: one bucket
    _learned(np.where(np.arange(N) % 2 == 0, -0.0, 0.0))      # signed zeros are distinct keys


def test_learned_fallbacks():
    need_gpu()
    rep = _learned(inputs.make_keys("mixture", 5000, seed=1))             # too small
    assert rep["fallback"] == 1
    rep = _learned(inputs.make_keys("mixture", N, seed=1), buffer_fraction=0.5)
    assert rep["fallback"] == 1
    rep = _learned(inputs.make_keys("mixture", N, seed=1), train_steps=0)  # no network
    assert rep["fallback"] == 0


N_HALF = (1 << 22) + 12347     # four leaves of about 2^20 keys, ragged


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("bf", [1.0, 0.5])
def test_misordered_partition_falls_back_to_plain_sort(bf, order):
    """A partition planted out of order (every key of bucket 2k sent to bucket
    2k+1 and the other way round): the bucket check fails, the plain merge sort
    re-sorts the whole array on the device, and the result is still exactly
    the oracle's stable sort -- with a report (which says so) and without one
    (no status error, no wrong order)."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    n = N if bf == 1.0 else N_HALF
    keys = inputs.make_keys("mixture", n, seed=31)
    g.gns_debug_learned_fault(g.FAULT_BUCKETS_SWAPPED)
    rep = _learned(keys, order=order, buffer_fraction=bf)
    assert rep["verify_failed"] == 1 and rep["fallback"] == 0, rep
    # no report requested: the same fallback, decided on the device
    g.gns_debug_learned_fault(g.FAULT_BUCKETS_SWAPPED)
    pay = inputs.index_payload(n)
    kt, pt = to_dev_keys(keys), to_dev_payload(pay)
    g.gns_learned_sort(kt, pt, order=order, buffer_fraction=bf)
    assert g.gns_stream_status() == 0
    want_k, want_p = oracle.stable_sort(keys, pay, oracle.DESC if order else oracle.ASC)
    assert_bitexact(kt.cpu().numpy(), pt.cpu().numpy().view(np.uint32), want_k, want_p)
    # the fault is consumed: the next call is clean
    assert _learned(keys, order=order, buffer_fraction=bf)["verify_failed"] == 0


def test_reversed_splitters_keep_the_partition_in_order():
    """Splitters reversed before the partition: a key's bucket comes from
    binary searches, whose outcome never decreases as the key grows whatever
    array is searched, so the buckets stay in order, the check passes and the
    result is exact without the fallback."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    keys = inputs.make_keys("mixture", N, seed=34)
    g.gns_debug_learned_fault(g.FAULT_SPLITTERS_REVERSED)
    rep = _learned(keys)
    assert rep["verify_failed"] == 0, rep


def test_garbage_network_weights_stay_exact():
    """NaN and +-1e30 weights make every splitter the same: one bucket takes
    nearly every key and is sorted by more merge levels of the same merge
    path.  The check passes (the splitters are in order) and the result is
    exact."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    keys = inputs.make_keys("mixture", N, seed=32)
    g.gns_debug_learned_fault(g.FAULT_GARBAGE_WEIGHTS)
    rep = _learned(keys)
    assert rep["verify_failed"] == 0 and rep["max_bucket"] > N // 2 and rep["overfull_buckets"] >= 1, rep
    g.gns_debug_learned_fault(g.FAULT_GARBAGE_WEIGHTS)
    assert _learned(keys, order=1, train_steps=0)["max_bucket"] > N // 2     # without training, too


def test_tiny_overfull_cap_stays_exact():
    """An overfull cap far below the mean bucket: every bucket counts as
    overfull and takes the merge path; the result is exact."""
    need_gpu()
    rep = _learned(inputs.make_keys("mixture", N, seed=33), overfull_factor=1e-3)
    assert rep["overfull_buckets"] == rep["nonempty_buckets"] > 1, rep


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("pattern", ["mixture", "ties", "permut", "asc_noise", "desc"])
def test_learned_half_buffer_exact(pattern, order):
    """The half-buffer form (four learned-sorted leaves of a two-level
    Frogsort1 tree, then two in-place merge levels) is bit-exact."""
    need_gpu()
    rep = _learned(inputs.make_keys(pattern, N_HALF, seed=21), order=order, buffer_fraction=0.5)
    assert rep["fallback"] == 0 and rep["nonempty_buckets"] >= 4


def test_learned_half_buffer_edges_and_ram():
    need_gpu()
    import paper_2402_01816_gb300 as g
    alpha = inputs.edge_alphabet()
    rng = np.random.default_rng(22)
    keys = np.concatenate([alpha[rng.integers(0, alpha.size, N_HALF // 2)], rng.normal(size=N_HALF - N_HALF // 2)])
    assert _learned(keys, order=0, buffer_fraction=0.75)["fallback"] == 0
    assert _learned(keys, order=1, with_payload=False, buffer_fraction=0.5)["fallback"] == 0
    assert _learned(np.full(N_HALF + 1, -2.5), buffer_fraction=0.5)["fallback"] == 0   # one value, odd n
    # below a half buffer the call is the plain (Frogsort2) sort
    assert _learned(inputs.make_keys("mixture", N_HALF, seed=23), buffer_fraction=0.4)["fallback"] == 1


def test_network_gain_over_first_stage():
    """What the trained network gains over the method without it (the
    first-stage quantile interpolation alone), on log-normal keys, where the
    density changes inside every first-stage interval: 256 Adam steps shrink
    the largest bucket to at most 0.85 of the first stage's (measured 0.69 to
    0.78 over five seeds), do not add overfull buckets, and lower the training
    loss against a short fit.  The result is exact either way."""
    need_gpu()
    rng = np.random.default_rng(100)
    logn = np.exp(rng.normal(0.0, 2.0, 1 << 22))
    first = _learned(logn, train_steps=0)
    short = _learned(logn, train_steps=32)
    trained = _learned(logn, train_steps=256)
    print("first stage only", first, "32 steps", short, "256 steps", trained)
    assert trained["max_bucket"] <= 0.85 * first["max_bucket"], (trained, first)
    assert trained["overfull_buckets"] <= first["overfull_buckets"], (trained, first)
    assert trained["final_loss"] < short["final_loss"], (trained, short)


def test_full_learned_workload():
    """2^28 float64 keys from the mixture: sorted, stable, a permutation, and
    sampled output positions from the oracle."""
    need_gpu()
    import paper_2402_01816_gb300 as g
    from tests.test_gpu_fullsize import check_sorted_stable
    n = 1 << 28
    keys = inputs.make_keys("mixture", n, seed=0)
    kt = to_dev_keys(keys)
    pt = to_dev_payload(inputs.index_payload(n))
    rep = g.gns_learned_sort(kt, pt, report=True)
    assert g.gns_stream_status() == 0 and rep["fallback"] == 0
    k_out = kt.cpu().numpy()
    p_out = pt.cpu().numpy().view(np.uint32)
    del kt, pt
    torch.cuda.empty_cache()
    check_sorted_stable(keys, k_out, p_out, samples=6)
