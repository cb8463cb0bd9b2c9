"""pe_loglike_batch_noalloc: the batched log-likelihood for callers that cannot allocate device
memory (for instance a sampler inside an application that has reserved the GPU's memory for its
own pool). It must give what pe_loglike_batch gives, call after call, using only the library's
fixed scratch array. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib as L
    B.build()
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    d = L.Detector(W.LISA, T, k0, nb)
    d.inject(W.theta_injection(T), W.MODE_ALL, W.normals(nb, 31))
    return torch, L, d, T


def _run(torch, L, d, th, noalloc):
    B = th.shape[0]
    tt = torch.tensor(th, device="cuda")
    logl = torch.empty(B, dtype=torch.float64, device="cuda")
    dhhh = torch.empty((B, 1, 3, 2), dtype=torch.float64, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    fn = L.pe_loglike_batch_noalloc if noalloc else L.pe_loglike_batch
    fn([d.handle], tt, B, W.MODE_ALL, logl, dhhh, st, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return logl.cpu().numpy(), dhhh.cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls(setup):
    """Two calls in a row (different batches) give pe_loglike_batch's results bit for bit: both run
    the same per-sub-tile partial sums in the same fixed reduction order, whatever launch choice
    each makes (the allocating entry point may use a tuned one)."""
    torch, L, d, T = setup
    for seed, B in ((401, 96), (402, 37)):
        th = W.draw_prior(B, seed, T)
        th[5, 1] = 0.5                                # one out-of-domain sample
        ref = _run(torch, L, d, th, noalloc=False)
        got = _run(torch, L, d, th, noalloc=True)
        np.testing.assert_array_equal(got[2], ref[2])
        assert np.all(np.isneginf(got[0][ref[2] != 0]))
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])


def test_noalloc_allocates_nothing_once_loaded(setup):
    """After a first call on the device (which loads the module holding the fixed array), a call
    changes neither the device's free memory nor torch's allocator, and it still runs when the
    caller has reserved all but a sliver of the device's memory for its own pool."""
    torch, L, d, T = setup
    th = torch.tensor(W.draw_prior(64, 404, T), device="cuda")
    logl = torch.empty(64, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    L.pe_loglike_batch_noalloc([d.handle], th, 64, W.MODE_ALL, logl, None, None, st)
    torch.cuda.synchronize()
    ref = logl.clone()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats().get("allocation.all.current", 0)
    L.pe_loglike_batch_noalloc([d.handle], th, 64, W.MODE_ALL, logl, None, None, st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.current", 0) == stats0
    # the caller's own pool takes all but 64 MiB of what is free
    hog = torch.empty(max(0, free0 - (64 << 20)), dtype=torch.uint8, device="cuda")
    try:
        logl.zero_()
        L.pe_loglike_batch_noalloc([d.handle], th, 64, W.MODE_ALL, logl, None, None, st)
        torch.cuda.synchronize()
        assert torch.equal(logl, ref)
    finally:
        del hog
        torch.cuda.empty_cache()


def test_noalloc_rejects_oversize_and_host_buffers(setup):
    torch, L, d, T = setup
    B = 20000                                         # about 116 MB of scratch on this grid
    th = torch.tensor(W.draw_prior(B, 3, T), device="cuda")
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    with pytest.raises(L.PeError) as e:
        L.pe_loglike_batch_noalloc([d.handle], th, B, W.MODE_ALL, out)
    assert e.value.status == L.PE_EINVAL and "scratch" in str(e.value)
    with pytest.raises(L.PeError) as e:
        L.pe_loglike_batch_noalloc([d.handle], W.draw_prior(4, 3, T), 4, W.MODE_ALL, np.zeros(4))
    assert e.value.status == L.PE_EINVAL


def test_noalloc_mixed_precision_matches_direct_call(setup):
    """The precision flag reaches the no-allocation entry point: same bits as pe_loglike_batch."""
    torch, L, d, T = setup
    th = W.draw_prior(50, 403, T)
    tt = torch.tensor(th, device="cuda")
    m = W.MODE_ALL | L.PE_PREC_MIXED
    outs = []
    for fn in (L.pe_loglike_batch, L.pe_loglike_batch_noalloc):
        logl = torch.empty(50, dtype=torch.float64, device="cuda")
        fn([d.handle], tt, 50, m, logl, None, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        outs.append(logl.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
