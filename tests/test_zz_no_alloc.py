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


def _ctx(kb, precision="fp64", ecut=5.0):
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, 91)
    ctx = paro.Context(lat, pos, ecut, 12, 8, precision, kpts=[(0.25, 0.0, -1 / 3)])
    ctx.set_local_pp(**inputs.LOCAL_PP)
    if kb:
        ctx.set_kb(inputs.KB_RC, inputs.kb_strengths(len(pos), 92))
    return ctx


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


# 5 Ha gives a 24^3 grid; at 10 Ha the grid is 32^3, where paro_apply_h takes the register-resident
# line FFTs while the allocation-free call keeps the shared-memory passes: both must agree
@pytest.mark.parametrize("ecut", [5.0, 10.0])
@pytest.mark.parametrize("kb", [False, True])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-6)])
def test_noalloc_matches_apply_h_on_two_calls_in_a_row(kb, dtype, tol, ecut):
    ctx = _ctx(kb, ecut=ecut)
    assert ctx.grid == ((24, 24, 24) if ecut == 5.0 else (32, 32, 32))
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


def _need_bytes(ctx, nb, elem):
    # the scratch formula the header states for paro_apply_h_noalloc
    def r(x):
        return (x + 255) // 256 * 256
    mil = ctx.miller()
    ncol = len({(int(a), int(b)) for a, b, _ in mil})
    p = 4 * ctx.n_atoms * nb
    need = r(nb * ctx.grid[2] * ncol * elem) + r(p * 16) + p * 16
    return need + (r(p * 8) if elem == 8 else 0)


@pytest.mark.parametrize("dtype,elem", [(torch.complex128, 16), (torch.complex64, 8)])
def test_noalloc_size_limit_follows_the_stated_formula(dtype, elem):
    from paper_1702_04045_gb300 import paro
    ctx = paro.context_from_config("si64_scf", "fp64")
    limit = 32 << 20
    nb = max(n for n in range(1, 145) if _need_bytes(ctx, n, elem) <= limit)
    psi = torch.from_numpy(inputs.start_vectors(nb + 1, ctx.npw(), 5)).to(dtype).cuda()
    out = torch.empty_like(psi)
    ctx.apply_h_noalloc(psi[:nb].contiguous(), out[:nb])          # the largest request that fits
    with pytest.raises(paro.ParoError) as e:                      # one band more does not
        ctx.apply_h_noalloc(psi, out)
    assert str(_need_bytes(ctx, nb + 1, elem)) in str(e.value)


def test_noalloc_binding_rejects_mismatched_output():
    from paper_1702_04045_gb300 import paro
    ctx = _ctx(True)
    psi = torch.zeros((3, ctx.npw()), dtype=torch.complex128, device="cuda")
    for bad in (torch.empty((2, ctx.npw()), dtype=torch.complex128, device="cuda"),
                torch.empty((3, ctx.npw()), dtype=torch.complex64, device="cuda"),
                torch.empty((ctx.npw(), 3), dtype=torch.complex128, device="cuda").t()):
        with pytest.raises(paro.ParoError):
            ctx.apply_h_noalloc(psi, bad)
    with pytest.raises(paro.ParoError):
        ctx.apply_h_noalloc(psi[:, :-1].contiguous(), torch.empty((3, ctx.npw() - 1), dtype=torch.complex128,
                                                                   device="cuda"))
