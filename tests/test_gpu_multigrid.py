"""Multigrid continuation on the GPU: gpe_interpolate against the oracle's
spectral interpolation (complex128: max|gpu - oracle| <= 1e-12 max|oracle|,
FP64 transforms of the same lines), exactness on band-limited fields, and a
multigrid solve whose finest answer the oracle verifies (||r||_inf < 1e-8)."""
import numpy as np
import pytest

from oracle import gpe_oracle as O
from paper_1611_02045_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G(built_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_02045_gb300 import gpe
    return gpe


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.complex128)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


CASES = [((32, 16), (64, 32)), ((64, 64), (128, 128)), ((256, 256), (512, 512)), ((16, 8, 16), (32, 16, 32)),
         ((64, 64), (128, 64)), ((8, 32), (8, 64)), ((8, 8), (16, 16)), ((32, 32, 32), (32, 32, 64))]


@pytest.mark.parametrize("nc,nf", CASES)
def test_interpolation_matches_oracle(G, nc, nf):
    L = tuple([6.0, 5.0, 4.0][: len(nc)])
    Vc = I.harmonic(nc, L)
    Vf = I.harmonic(nf, L)
    pc = O.Problem(nc, L, 10.0, 0.3, Vc)
    pf = O.Problem(nf, L, 10.0, 0.3, Vf)
    fc = I.random_field(71, nc, L)
    want = O.interpolate(pc, fc, pf)
    with G.Context(nc, L, 10.0, 0.3, Vc, prec=G.GPE_FP64) as cc, G.Context(nf, L, 10.0, 0.3, Vf, prec=G.GPE_FP64) as cf:
        out = torch.empty(want.shape, dtype=torch.complex128, device="cuda")
        cc.interpolate_to(cf, dev(fc), out)
        got = host(out)
        host_out = np.zeros(want.shape, dtype=np.complex128)
        cc.interpolate_to(cf, fc, host_out)  # host in, host out
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert np.array_equal(host_out, got)


def test_interpolation_is_exact_on_band_limited_fields(G):
    nc, nf, L = (32, 32), (64, 64), (6.0, 6.0)
    m_c, m_f = I.mesh(nc, L), I.mesh(nf, L)

    def field(m):
        return (np.exp(1j * (3 * np.pi / L[0] * (m[0] + L[0]) - 5 * np.pi / L[1] * (m[1] + L[1])))
                + 0.5 * np.cos(16 * np.pi / L[0] * (m[0] + L[0])))

    with G.Context(nc, L, 1.0, 0.0, I.harmonic(nc, L), prec=G.GPE_FP64) as cc, \
            G.Context(nf, L, 1.0, 0.0, I.harmonic(nf, L), prec=G.GPE_FP64) as cf:
        out = torch.empty((64, 64), dtype=torch.complex128, device="cuda")
        cc.interpolate_to(cf, dev(field(m_c)), out)
    assert np.max(np.abs(host(out) - field(m_f))) < 1e-12


def test_interpolation_rejects_mismatched_grids(G):
    with G.Context((32, 32), (6.0, 6.0), 1.0, 0.0, I.harmonic((32, 32), (6.0, 6.0))) as cc, \
            G.Context((128, 128), (6.0, 6.0), 1.0, 0.0, I.harmonic((128, 128), (6.0, 6.0))) as c4, \
            G.Context((64, 64), (7.0, 6.0), 1.0, 0.0, I.harmonic((64, 64), (7.0, 6.0))) as cl:
        x = torch.zeros((32, 32), dtype=torch.complex128, device="cuda")
        y = torch.zeros((128, 128), dtype=torch.complex128, device="cuda")
        z = torch.zeros((64, 64), dtype=torch.complex128, device="cuda")
        with pytest.raises(G.GpeError):
            cc.interpolate_to(c4, x, y)  # factor 4 in one step
        with pytest.raises(G.GpeError):
            cc.interpolate_to(cl, x, z)  # different domain


def test_multigrid_solve_reaches_a_verified_ground_state(G):
    """64^2 -> 128^2 -> 256^2 on the fast-rotation trap of the 256^2 workload,
    from the Thomas-Fermi state; the finest answer is checked by the oracle."""
    from paper_1611_02045_gb300.multigrid import multigrid_solve
    w = I.workload("fast256_2d")
    phi, reps = multigrid_solve([64, 128, 256], w["L"], w["eta"], w["omega"], lambda n, L: I.harmonic(n, L))
    assert [r["status"] for r in reps] == [G.GPE_OK] * 3, reps
    po = O.Problem(w["n"], w["L"], w["eta"], w["omega"], w["V"])
    ph = host(phi)
    lam = O.chemical_potential(po, ph)
    assert np.max(np.abs(O.apply_H(po, ph, ph) - lam * ph)) < 1e-8
    assert abs(O.energy(po, ph) - reps[-1]["E"]) <= 1e-12 * abs(reps[-1]["E"])
    assert abs(O.norm(po, ph) - 1.0) < 1e-12
