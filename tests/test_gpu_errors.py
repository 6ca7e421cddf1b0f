"""Error paths through the C ABI: failures injected on the host (LEV_FAULT), malformed CSR input,
and a device wait that runs out.

Nothing here faults the GPU: LEV_FAULT makes the library report a failed allocation, a failed
launch or an expired device wait at its host-side checks, and the CSR check rejects malformed row
pointers before any kernel reads the column or value arrays. LEV_FAULT=pivwait has the pivoted
Cholesky withhold one published pivot column, so that the other CTAs' bounded waits for it (about
a second) really run out on the device: the kernels record the timeout in the status word and
return, with no trap. After each error the same handle must serve a clean call whose result is
bit-identical to that of a fresh handle, and the device status word must read 0.
"""
import numpy as np
import pytest

import workloads as W

from ._gpu import lev_module, to_dev

pytestmark = pytest.mark.gpu

CFG = dict(s=4096, m=192, k=32, tau=1e-6, seed=8, sketch_prec="bf16x3", final_prec="bf16x3")


@pytest.fixture(scope="module")
def L():
    return lev_module()


def _reference_theta(L, A):
    import torch
    h = L.Handle(0)
    try:
        th = torch.empty(A.shape[0], device="cuda")
        L.lev_estimate_dense(h, A, L.make_params(**CFG), th)
        return th
    finally:
        h.close()


@pytest.mark.parametrize("fault,code", [("alloc", "LEV_ENOMEM"), ("launch", "LEV_ECUDA"),
                                        ("timeout", "LEV_ETIMEOUT")])
def test_injected_failure_then_clean_call(L, monkeypatch, fault, code):
    import torch
    A = to_dev(W.dense_gaussian(6000, 48, 3).astype(np.float32))
    want = _reference_theta(L, A)
    h = L.Handle(0)
    try:
        th = torch.empty(6000, device="cuda")
        monkeypatch.setenv("LEV_FAULT", fault)
        with pytest.raises(L.LevError) as e:
            L.lev_estimate_dense(h, A, L.make_params(**CFG), th)
        assert e.value.code == getattr(L, code)
        assert "LEV_FAULT=" + fault in str(e.value)
        monkeypatch.delenv("LEV_FAULT")
        assert L.lev_estimate_dense(h, A, L.make_params(**CFG), th) == 48
        assert torch.equal(th, want)
        assert L.lev_device_status(h) == 0
    finally:
        h.close()


def _csr(n=3000, d=40):
    C = W.csr_uniform(n, d, nnz_per_row=6, heavy_frac=0.0, seed=9)
    return C, C.row_ptr.copy()


@pytest.mark.parametrize("defect", ["first", "decreasing", "last"])
def test_malformed_csr_is_rejected_before_any_kernel_reads_it(L, defect):
    import torch
    C, rp = _csr()
    n, d = C.shape
    if defect == "first":
        rp = rp + 1                                     # row_ptr[0] = 1 (and row_ptr[n] = nnz + 1)
        word = "row_ptr[0] != 0"
    elif defect == "decreasing":
        rp[n // 2] = rp[n // 2 + 1] + 5                 # one row pointer past the next one
        word = "row_ptr decreases"
    else:
        rp[n] = rp[n] - 3                               # row_ptr[n] != nnz
        word = "row_ptr[n] != nnz"
    h = L.Handle(0)
    try:
        rpd, cl, vl = to_dev(rp), to_dev(C.col), to_dev(C.val)
        theta = torch.empty(n, device="cuda")
        p = L.make_params(s=1024, m=160, k=16, tau=1e-5, seed=2)
        calls = [
            lambda: L.lev_estimate_csr(h, rpd, cl, vl, n, d, p, theta),
            lambda: L.lev_sketch_csr(h, rpd, cl, vl, n, d, p, torch.empty((160, d), device="cuda")),
            lambda: L.lev_final_csr(h, rpd, cl, vl, n, d, torch.zeros((d, 16), device="cuda"), "fp32", theta),
            lambda: L.lev_exact_reference_csr(h, rpd, cl, vl, n, d, 1e-5, theta),
        ]
        for call in calls:
            with pytest.raises(L.LevError) as e:
                call()
            assert e.value.code == L.LEV_EINVAL
            assert word in str(e.value)
        # the same handle then serves a well-formed call, checked or vouched for by the caller
        good = to_dev(C.row_ptr)
        r1 = L.lev_estimate_csr(h, good, cl, vl, n, d, p, theta)
        t1 = theta.clone()
        pu = L.make_params(s=1024, m=160, k=16, tau=1e-5, seed=2)
        pu.flags |= L.LEV_CSR_UNCHECKED
        r2 = L.lev_estimate_csr(h, good, cl, vl, n, d, pu, theta)
        assert r1 == r2 == d and torch.equal(t1, theta)
        assert L.lev_device_status(h) == 0
    finally:
        h.close()


def _sketch(m, d, r, seed):
    rs = np.random.default_rng(seed)
    X = rs.standard_normal((m, r)) @ rs.standard_normal((r, d))
    X *= np.exp(rs.standard_normal(d))[None, :]
    return X.astype(np.float32)


@pytest.mark.parametrize("m,d,r", [(192, 48, 40), (1024, 256, 200), (2048, 512, 450)])
def test_device_wait_runs_out_then_clean_call(L, monkeypatch, m, d, r):
    """The pivoted Cholesky of the Gram route (the cluster form up to d = 256, the grid form above)
    never publishes its second pivot column: the waits for it expire on the device, the call reports
    LEV_ETIMEOUT, and the handle then factors the same sketch exactly as a fresh handle does."""
    import torch
    At = to_dev(_sketch(m, d, r, seed=d))
    tau = 1e-5

    def rrqr(h):
        perm = torch.empty(d, dtype=torch.int32, device="cuda")
        R = torch.empty((d, d), dtype=torch.float64, device="cuda")
        return L.lev_rrqr(h, At, tau, perm, R), perm, R

    h0 = L.Handle(0)
    try:
        r0, p0, R0 = rrqr(h0)
    finally:
        h0.close()
    assert r0 == r
    h = L.Handle(0)
    try:
        monkeypatch.setenv("LEV_FAULT", "pivwait")
        with pytest.raises(L.LevError) as e:
            rrqr(h)
        assert e.value.code == L.LEV_ETIMEOUT
        assert "bounded device wait" in str(e.value)
        monkeypatch.delenv("LEV_FAULT")
        assert L.lev_device_status(h) == 0
        r1, p1, R1 = rrqr(h)
        assert r1 == r0
        assert torch.equal(p1, p0) and torch.equal(R1, R0)
        assert L.lev_device_status(h) == 0
    finally:
        h.close()

