"""gpe_apply_H_noalloc: the allocation-free H_phi f for callers that cannot
allocate device memory (it keeps its scratch in a fixed static device array).

Checked through the C ABI against gpe_apply_H (which uses a context's
allocated workspace) on two calls in a row with different inputs, so that
anything left in the shared scratch by the first call would show in the
second.  Collected last on purpose (file name), and independent of the other
test files' state."""
import ctypes as C

import numpy as np
import pytest

from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G(built_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_02045_gb300 import gpe
    L = gpe.lib()
    L.gpe_apply_H_noalloc.argtypes = [C.POINTER(gpe.gpe_problem), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_char_p, C.c_size_t]
    L.gpe_apply_H_noalloc.restype = C.c_int
    return gpe


def problem(G, n, L, eta, omega, prec):
    p = G.gpe_problem()
    p.dim = len(n)
    for i in range(3):
        p.n[i] = n[i] if i < len(n) else 1
        p.L[i] = L[i] if i < len(L) else 1.0
    p.eta, p.omega, p.prec = eta, omega, prec
    return p


def noalloc(G, p, V, phi, f, out):
    buf = C.create_string_buffer(256)
    s = G.lib().gpe_apply_H_noalloc(C.byref(p), V.data_ptr(), phi.data_ptr(), f.data_ptr(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream, buf, 256)
    return s, buf.value.decode()


@pytest.mark.parametrize("n,L", [((64, 64), (8.0, 8.0)), ((256, 128), (16.0, 8.0)), ((32, 32, 32), (6.0, 6.0, 6.0))])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_noalloc_matches_apply_H_on_two_calls(G, n, L, prec):
    eta, om = 37.0, 0.7
    V = I.harmonic(n, L)
    cdt = torch.complex128 if prec == 0 else torch.complex64
    rdt = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 2e-5
    Vd = torch.from_numpy(V.copy()).to("cuda", rdt)
    p = problem(G, n, L, eta, om, prec)
    with G.Context(n, L, eta, om, V, prec=prec) as ctx:
        for seed in (1, 5):
            phi = torch.from_numpy(I.random_field(seed, n, L)).to("cuda", cdt)
            f = torch.from_numpy(I.random_field(seed + 1, n, L)).to("cuda", cdt)
            want = torch.empty_like(f)
            ctx.apply_H(phi, f, want)
            got = torch.full_like(f, float("nan"))
            s, msg = noalloc(G, p, Vd, phi, f, got)
            assert s == G.GPE_OK, msg
            torch.cuda.synchronize()
            w = want.cpu().numpy()
            assert np.all(np.isfinite(got.cpu().numpy()))
            assert np.max(np.abs(got.cpu().numpy() - w)) <= tol * np.max(np.abs(w))


def test_noalloc_rejects_grids_beyond_its_scratch(G):
    n, L = (512, 512, 8), (8.0, 8.0, 8.0)  # 2^21 complex128 points: 32 MiB > 16 MiB
    p = problem(G, n, L, 1.0, 0.0, 0)
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    s, msg = noalloc(G, p, x, x, x, x)
    assert s == G.GPE_ERR_UNSUPPORTED
    assert "limit" in msg
    p.n[0] = 12
    s, msg = noalloc(G, p, x, x, x, x)
    assert s == G.GPE_ERR_ARG and msg


def test_noalloc_rejects_grids_beyond_its_block_limit_before_any_work(G):
    """512 x 8 x 512 complex64 fits the 16 MiB field (2^21 points) but its y
    pass needs 16384 thread blocks, more than the 8192 the scratch partials
    hold: rejected up front, out left as it was."""
    n, L = (512, 8, 512), (8.0, 8.0, 8.0)
    p = problem(G, n, L, 1.0, 0.0, 1)
    N = 512 * 8 * 512
    V = torch.zeros(N, dtype=torch.float32, device="cuda")
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    out = torch.full((N,), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")
    s, msg = noalloc(G, p, V, x, x, out)
    assert s == G.GPE_ERR_UNSUPPORTED, msg
    assert "thread blocks" in msg
    torch.cuda.synchronize()
    assert bool(torch.all(out == (7.0 + 3.0j)))
