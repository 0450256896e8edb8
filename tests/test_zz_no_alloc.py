"""dda_matvec_noalloc: the product without any allocation, for callers that cannot
allocate device memory (a fixed budget owned by another allocator, or loops
where cudaMalloc/cudaFree would synchronize the device).

It must give the same A.P as dda_matvec, call after call (the fixed scratch is
shared and keeps the previous call's contents), and refuse requests larger
than its fixed 32 MiB scratch.  The file sorts last so that a run stopping at
the first failure has run every other test first.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


# (workload, RHS per call for complex64, for complex128): the 64x48x32 grid needs 9.4 MB of
# complex64 scratch per RHS on its 3-pass schedule and 18.9 MB of complex128 scratch on its 5-pass one,
# so one complex128 RHS fits the fixed 32 MiB and two do not.
CASES = [(W.Workload("ell_odd", "ELLIPSOID", (7, 5, 9), 1.5 + 0.1j, 2.0, "GKDLDR", W.uniform_orientations(2, 11)),
          4, 4),
         (W.ELLIPSOID64, 2, 1)]


@pytest.mark.parametrize("w,nr64,nr128", CASES, ids=["small_4rhs", "ellipsoid64"])
def test_noalloc_product_matches_allocating_product_twice(D, w, nr64, nr128):
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    for dt, tol, nr in ((torch.complex64, 1e-5, nr64), (torch.complex128, 1e-12, nr128)):
        p = torch.from_numpy(W.seeded_vector((nr, 3, ctx.n), 41)).to(dt).cuda()
        ref = torch.empty_like(p)
        ctx.dda_matvec(p, ref, nrhs=nr)
        torch.cuda.synchronize()
        ref_np = ref.cpu().numpy().astype(np.complex128)
        for call in range(2):
            out = torch.full_like(p, float("nan"))
            ctx.dda_matvec_noalloc(p, out, nrhs=nr)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.complex128)
            assert np.isfinite(got).all()
            err = np.linalg.norm(got - ref_np) / np.linalg.norm(ref_np)
            assert err <= tol, (dt, call, err)
    if w is W.ELLIPSOID64:  # two complex128 RHS exceed the fixed scratch
        p2 = torch.zeros((2, 3, ctx.n), dtype=torch.complex128, device="cuda")
        with pytest.raises(D.DDAError) as ei:
            ctx.dda_matvec_noalloc(p2, torch.empty_like(p2), nrhs=2)
        assert ei.value.status == D.DDA_EINVAL


def test_noalloc_first_on_a_fresh_context_allocates_nothing(D):
    """On a freshly set-up context whose first product is dda_matvec_noalloc: device free memory is
    the same before and after a call (outputs allocated beforehand), and only then is the result
    compared with dda_matvec's."""
    w = W.Workload("ell_fresh", "ELLIPSOID", (9, 7, 11), 1.4 + 0.2j, 2.5, "LATTDR", W.uniform_orientations(2, 23))
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    for dt, tol in ((torch.complex64, 1e-5), (torch.complex128, 1e-12)):
        p = torch.from_numpy(W.seeded_vector((ctx.nrhs, 3, ctx.n), 43)).to(dt).cuda()
        outs = [torch.full_like(p, float("nan")) for _ in range(3)]
        torch.cuda.synchronize()
        ctx.dda_matvec_noalloc(p, outs[0])  # first product of this context
        torch.cuda.synchronize()
        for k in (1, 2):
            free0 = torch.cuda.mem_get_info()[0]
            ctx.dda_matvec_noalloc(p, outs[k])
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, (dt, k)
        ref = torch.empty_like(p)
        ctx.dda_matvec(p, ref)
        torch.cuda.synchronize()
        ref_np = ref.cpu().numpy().astype(np.complex128)
        for k in range(3):
            got = outs[k].cpu().numpy().astype(np.complex128)
            assert np.isfinite(got).all()
            assert np.linalg.norm(got - ref_np) / np.linalg.norm(ref_np) <= tol, (dt, k)


def test_noalloc_rejects_requests_beyond_the_fixed_scratch(D):
    ctx = D.Context(0)
    D.setup_workload(ctx, W.PRISM48)  # 128 RHS x 5.3 MB of complex64 scratch each
    p = torch.zeros((ctx.nrhs, 3, ctx.n), dtype=torch.complex64, device="cuda")
    ap = torch.empty_like(p)
    with pytest.raises(D.DDAError) as ei:
        ctx.dda_matvec_noalloc(p, ap)
    assert ei.value.status == D.DDA_EINVAL
    assert "fixed limit" in str(ei.value)
    ctx.dda_matvec_noalloc(p, ap, nrhs=4)  # a few RHS fit
    torch.cuda.synchronize()
    assert torch.count_nonzero(ap[:4]).item() == 0
