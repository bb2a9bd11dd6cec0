"""The allocation-free H psi entry point (paro_apply_h_noalloc) against paro_apply_h.

paro_apply_h_noalloc serves callers that cannot let the library allocate device memory mid-call
(applications that run all device memory through their own fixed pool, or that must keep the
device-wide synchronisation of cudaMalloc/cudaFree out of a tight loop); its scratch is one fixed
32 MiB device array shared by every call. These tests call it twice in a row with different inputs,
so a result that leaned on the previous call's scratch contents would show up, and check that a
request beyond the fixed size is refused with a clear error. This file is collected last.
"""
import numpy as np
import pytest

from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx(kb, precision="fp64"):
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, 91)
    ctx = paro.Context(lat, pos, 5.0, 12, 8, precision, kpts=[(0.25, 0.0, -1 / 3)])
    ctx.set_local_pp(**inputs.LOCAL_PP)
    if kb:
        ctx.set_kb(inputs.KB_RC, inputs.kb_strengths(len(pos), 92))
    return ctx


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("kb", [False, True])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-6)])
def test_noalloc_matches_apply_h_on_two_calls_in_a_row(kb, dtype, tol):
    ctx = _ctx(kb)
    npw = ctx.npw()
    rng = np.random.default_rng(17)
    outs = []
    for nb in (7, 12):  # two calls in a row, different band counts and inputs
        psi = torch.from_numpy(rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))).to(dtype).cuda()
        ref = ctx.apply_h(psi)
        out = torch.full_like(psi, float("nan"))
        ctx.apply_h_noalloc(psi, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out.real).all() and torch.isfinite(out.imag).all()
        assert _rel(out, ref) < tol
        outs.append(out)
    assert outs[0].shape != outs[1].shape


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_1702_04045_gb300 import paro
    ctx = paro.context_from_config("si64_scf", "fp64")
    psi = torch.zeros((144, ctx.npw()), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(psi)
    with pytest.raises(paro.ParoError) as e:
        ctx.apply_h_noalloc(psi, out)
    assert e.value.status == paro.PARO_ERR_ARG
    assert "32 MiB" in str(e.value)
    # a request that fits still works on the same context afterwards
    small = torch.from_numpy(inputs.start_vectors(2, ctx.npw(), 3)).cuda()
    ref = ctx.apply_h(small)
    got = torch.empty_like(small)
    ctx.apply_h_noalloc(small, got)
    assert _rel(got, ref) < 1e-12
