"""Failure detection without a GPU fault: every host wait of the library is bounded (PE_ETIMEOUT,
the work stays queued and completes), checked with a short limit on a normal, short call."""
import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Lb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2602_12011_gb300 import build as B
    from paper_2602_12011_gb300 import _lib
    B.build()
    _lib.lib()
    return _lib


def test_host_wait_times_out_and_the_work_completes(Lb):
    """With a 1 microsecond limit, a call that returns into pinned host memory gives PE_ETIMEOUT
    while its kernels are still running; after a stream synchronise the outputs equal those of the
    same call under the default limit, and the context keeps working."""
    import torch
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    d = Lb.Detector(W.LISA, T, k0, nb)
    d.inject(W.theta_injection(T), W.MODE_ALL, W.normals(nb, 1))
    th = torch.tensor(W.draw_prior(256, 7, T)).pin_memory()
    ref = Lb.loglike([d], th.numpy(), W.MODE_ALL)["logl"]
    out = torch.zeros(256, dtype=torch.float64).pin_memory()
    st = torch.cuda.current_stream()
    old = Lb.pe_get_wait_limit()
    Lb.pe_set_wait_limit(1e-6)
    try:
        with pytest.raises(Lb.PeError) as e:
            Lb.pe_loglike_batch([d.handle], th, 256, W.MODE_ALL, out, None, None, st)
        assert e.value.status == Lb.PE_ETIMEOUT
    finally:
        Lb.pe_set_wait_limit(old)
    st.synchronize()
    assert np.array_equal(out.numpy(), ref)
    again = Lb.loglike([d], th.numpy(), W.MODE_ALL)["logl"]
    assert np.array_equal(again, ref)
    d.close()


# ---- the test build: host-side fault injection and index checks (include/pespace_gb300_test.h)
@pytest.fixture(scope="module")
def TL(Lb):
    from paper_2602_12011_gb300 import build as B
    tl = Lb.load(B.build(variant="test"))
    prev = Lb.swap_library(tl)
    try:
        yield tl
    finally:
        tl.pe_test_fault_arm(-1, 0)
        Lb.swap_library(prev)


def _small_setup(Lb):
    T = 2.0 ** 15
    k0, nb = W.grid(T)
    th = W.draw_prior(5, 17, T)
    th[0] = W.theta_injection(T)
    data = np.zeros((3, nb), dtype=np.complex128)
    return T, k0, nb, th, data


def _scenarios(Lb):
    """Each scenario runs one entry point (or a create/use/destroy cycle) on a small case and closes
    every handle it made, whether the entry point succeeded or not."""
    import torch
    T, k0, nb, th, data = _small_setup(Lb)
    nrm = W.normals(nb, 3)

    def lifecycle():
        d = Lb.Detector(W.LISA, T, k0, nb)
        try:
            d.set_data(data)
            d.inject(th[0], W.MODE_ALL, nrm)
            return d.data_norm()
        finally:
            d.close()

    def with_det(fn):
        def run():
            d = Lb.Detector(W.LISA, T, k0, nb)
            try:
                d.inject(th[0], W.MODE_ALL, nrm)
                return fn(d)
            finally:
                d.close()
        return run

    def plan(d):
        p = Lb.Plan([d], th.shape[0], W.MODE_ALL, theta=torch.tensor(th, device="cuda"), autotune=False)
        try:
            p.launch()
            torch.cuda.synchronize()
            return p.logl.cpu().numpy()
        finally:
            p.close()

    def hetero(d):
        h = Lb.Hetero(d, th[0], W.MODE_ALL, nbins_coarse=32)
        try:
            return Lb.hetero_loglike([h], th)["logl"]
        finally:
            h.close()

    def surrogate():
        s = Lb.Surrogate(seed=5)
        try:
            return s.predict(torch.tensor(th, device="cuda")).cpu().numpy()
        finally:
            s.close()

    return {
        "detector": lifecycle,
        "loglike_host": with_det(lambda d: Lb.loglike([d], th, W.MODE_ALL, dhhh=True)["logl"]),
        "loglike_device": with_det(lambda d: Lb.loglike([d], torch.tensor(th, device="cuda"), W.MODE_ALL)["logl"]
                                   .cpu().numpy()),
        "grad": with_det(lambda d: Lb.loglike_grad([d], th, W.MODE_ALL)["grad"]),
        "fisher": with_det(lambda d: Lb.fisher([d], th[:2], W.MODE_ALL)),
        "plan": with_det(plan),
        "hetero": with_det(hetero),
        "surrogate": surrogate,
    }


@pytest.mark.parametrize("name", ["detector", "loglike_host", "loglike_device", "grad", "fisher", "plan", "hetero",
                                  "surrogate"])
def test_every_injected_fault_returns_a_status_and_leaks_nothing(Lb, TL, name):
    """For each entry point: every device allocation, upload and launch it makes is failed in turn
    (one per call). Each such call returns a PE_* error with a message, the test build counts no
    device allocation left behind once the stream work has drained, and the next undisturbed call
    gives the same result as before."""
    import torch
    run = _scenarios(Lb)[name]
    TL.pe_test_fault_arm(-1, 0)
    live0 = TL.pe_test_live_allocations()
    ref = run()
    torch.cuda.synchronize()
    counts = [TL.pe_test_fault_count(k) for k in range(3)]
    assert TL.pe_test_live_allocations() == live0
    assert counts[0] > 0 and counts[2] > 0, counts
    for kind in range(3):
        for nth in range(1, counts[kind] + 1):
            TL.pe_test_fault_arm(kind, nth)
            with pytest.raises(Lb.PeError) as e:
                run()
            assert e.value.status in (Lb.PE_ENOMEM, Lb.PE_ECUDA, Lb.PE_EINVAL), (kind, nth, e.value)
            assert TL.pe_test_fault_fired() == 1, (kind, nth)
            torch.cuda.synchronize()
            assert TL.pe_test_live_allocations() == live0, (name, kind, nth, str(e.value))
    TL.pe_test_fault_arm(-1, 0)
    again = run()
    assert np.array_equal(np.asarray(again), np.asarray(ref))
    assert TL.pe_test_checked_take() == 0


def test_checked_build_matches_the_product_bitwise(Lb, TL):
    """The index-checked kernels of the test build give bit-identical log L, <d|h>, <h|h>, gradient
    and Fisher on small ragged cases (FP64 and mixed, one and three detectors), and no check fires."""
    prev = Lb.swap_library(Lb.load(Lb.LIB_PATH))
    try:
        res_p = _checked_cases(Lb)
    finally:
        Lb.swap_library(prev)
    res_t = _checked_cases(Lb)
    for k in res_p:
        assert np.array_equal(res_p[k], res_t[k]), k
    assert TL.pe_test_checked_take() == 0


def _checked_cases(Lb):
    out = {}
    dets = []
    for det, T in ((W.LISA, 2.0 ** 16), (W.TAIJI, 2.0 ** 15), (W.TIANQIN, 2.0 ** 14)):
        k0, nb = W.grid(T)
        d = Lb.Detector(det, T, k0, nb)
        d.inject(W.theta_injection(2.0 ** 14), W.MODE_ALL, W.normals(nb, 9))
        dets.append(d)
    th = W.draw_prior(9, 23, 2.0 ** 14)
    try:
        for tag, ds in (("one", dets[:1]), ("net", dets)):
            for prec in (0, Lb.PE_PREC_MIXED):
                g = Lb.loglike(ds, th, W.MODE_ALL | prec, dhhh=True)
                out["ll_%s_%d" % (tag, prec)] = g["logl"]
                out["dhhh_%s_%d" % (tag, prec)] = g["dhhh"]
                out["grad_%s_%d" % (tag, prec)] = Lb.loglike_grad(ds, th[:4], W.MODE_ALL | prec)["grad"]
            out["fisher_%s" % tag] = Lb.fisher(ds, th[:2], W.MODE_ALL)
    finally:
        for d in dets:
            d.close()
    return out
