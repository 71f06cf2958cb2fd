"""The allocation-free operator application against the context-based one.

psfd_apply_fp32_static exists for callers that cannot call cudaMalloc (device memory
fixed at start-up, or a host allocator that owns the device): it needs no context and
keeps every intermediate in the library's static device scratch. Its output must equal
psfd_apply's FP32 output within the FP32 operator tolerance of the parity tests, on
consecutive calls that reuse the scratch left behind by the previous call (grids that take
the fused and the split plane kernels, with, without and with an irregular stack), and the
oracle's FP64 operator within the same tolerance.

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2606_25541_b300 import layouts

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 3e-5  # FP32 operator tolerance of tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def psfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25541_b300 import psfd as m
    m.load()
    return m


def _grid(psfd, p):
    return psfd.make_grid(p.nx, p.ny, p.nslab, p.nf, p.dx, p.dy, p.dz, p.wavelength, p.eps_bg)


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _graded_stack():
    """Twelve layers of twelve different indices (more distinct media than the by-value tables hold)."""
    n = np.array([0.9 + 0.01 * k + (0.002 + 0.0005 * k) * 1j for k in range(12)], np.complex128)
    return n, np.full(12, 3.1), 0.97 + 0.02j


def test_static_apply_matches_context_apply_on_consecutive_calls(psfd):
    cases = [
        (layouts.line_space_clip(), 5, 1),
        (layouts.small_clip(nx=32, ny=32, nslab=7, dx=2.0, dz=1.5, seed=4, stack=layouts.ru_mosi_stack(10)), 0, 2),
        (layouts.line_space_clip(), 16, 3),
        # split planes (row and column passes), 43.5 MB of the 48 MiB scratch
        (layouts.small_clip(nx=256, ny=256, nslab=16, dx=1.0, dz=1.0, seed=6, stack=layouts.ru_mosi_stack(40)), 0, 4),
        # no stack at all (n_layers = 0, the substrate alone)
        (layouts.small_clip(nx=64, ny=64, nslab=9, dx=2.0, dz=1.0, seed=7, stack=layouts.empty_stack(1.0 + 0.1j)), 0, 5),
        # a stack too varied to pass by value: copied into the scratch
        (layouts.small_clip(nx=32, ny=32, nslab=5, dx=2.0, dz=1.5, seed=8, stack=_graded_stack()), 0, 6),
    ]
    for prob, i, seed in cases:
        eps = torch.from_numpy(prob.eps).cuda()
        u = torch.tensor(layouts.random_field((3, prob.nslab, prob.ny, prob.nx), seed=seed), dtype=torch.complex64,
                         device="cuda")
        out_static = torch.full_like(u, float("nan"))
        st = psfd.apply_fp32_static(_grid(psfd, prob), prob.n_layers, prob.d_layers, prob.n_sub,
                                    prob.theta_deg[i], prob.phi_deg[i], eps, u, out_static)
        assert st == psfd.OK, psfd.strerror(st)
        one = prob.with_illumination(prob.theta_deg[[i]], prob.phi_deg[[i]], prob.pol[[i]])
        s = psfd.Solver.from_problem(one, psfd.FP32_REFINED)
        out_ref = torch.empty_like(u)
        s.apply(u[None], out_ref[None])
        torch.cuda.synchronize()
        assert _rel(out_static, out_ref) < TOL
        assert _rel(u - out_static, u - out_ref) < TOL
        s.close()


def test_static_apply_matches_the_oracle(psfd):
    """The same entry point against the FP64 oracle's operator (Sec. 3, Eq. (18) with the
    reflection of Eq. (9)), on a clip small enough for the oracle."""
    import oracle
    prob = layouts.small_clip(nx=32, ny=32, nslab=7, dx=2.0, dz=1.5, seed=4, stack=layouts.ru_mosi_stack(40),
                              theta=(6.0,), phi=(30.0,), pol=(1,))
    u64 = layouts.random_field((3, prob.nslab, prob.ny, prob.nx), seed=9)
    u = torch.tensor(u64, dtype=torch.complex64, device="cuda")
    out = torch.full_like(u, float("nan"))
    for _ in range(2):
        st = psfd.apply_fp32_static(_grid(psfd, prob), prob.n_layers, prob.d_layers, prob.n_sub,
                                    prob.theta_deg[0], prob.phi_deg[0], torch.from_numpy(prob.eps).cuda(), u, out)
        assert st == psfd.OK, psfd.strerror(st)
        torch.cuda.synchronize()
        ref = oracle.apply_operator(oracle.setup_rhs(prob, 0), u.cpu().numpy().astype(np.complex128))
        got = out.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) < TOL * np.linalg.norm(ref)


def test_static_apply_rejects_grids_beyond_its_scratch(psfd):
    g = psfd.make_grid(256, 256, 60, 128, 1.0, 1.0, 1.0, 13.5)
    dummy = torch.zeros(4, dtype=torch.complex128, device="cuda")
    n, d, ns = layouts.ru_mosi_stack(2)
    st = psfd.apply_fp32_static(g, n, d, ns, 6.0, 0.0, dummy, dummy, dummy)
    assert st == psfd.E_BUDGET
    assert bool(torch.all(dummy == 0))
