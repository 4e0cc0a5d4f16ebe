"""hmg_line_smooth_noalloc: the line-smoothing sweeps for callers that cannot allocate
device memory during the call (their memory belongs to another allocator, or a budget fixed
at start-up, or cudaMalloc's device synchronisation is unaffordable). It must give what
hmg_line_smooth gives, call after call, while taking its second vector from an array built
into the library instead of the context's workspace.

Collected last (file name) so that a run stopping at the first failure has already run every
other test; it builds its own context, so it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2210_11797_gb300 import inputs as I


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64)).cuda()


@pytest.mark.parametrize("nsweeps", [1, 2])
def test_noalloc_line_smooth_matches_line_smooth(nsweeps):
    from paper_2210_11797_gb300 import hmg
    w = I.cubed_sphere(12, 30)                    # 314,496 trace unknowns, within the 1,048,576 limit
    gpu = hmg.Solver(w.hier, w.coeffs, tol=w.tol)
    L = hmg.lib()
    rng = np.random.default_rng(11)
    lam0 = rng.standard_normal(gpu.ntrace)
    b = _cuda(gpu.apply_trace(_cuda(rng.standard_normal(gpu.ntrace))).cpu().numpy())
    ref = _cuda(lam0)
    gpu.line_smooth(b, ref, nsweeps)              # the existing entry point
    ref = ref.cpu().numpy()
    for call in range(2):                         # two calls in a row share the built-in array
        lam = _cuda(lam0)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = L.hmg_line_smooth_noalloc(gpu.ctx, ctypes.c_void_p(b.data_ptr()),
                                       ctypes.c_void_p(lam.data_ptr()), nsweeps)
        assert st == 0, L.hmg_last_error(gpu.ctx).decode()
        # the array was placed when hmg_assemble_trace looked up its address, so the call
        # itself takes no device memory, the first call included
        assert torch.cuda.mem_get_info()[0] == free_before, call
        got = lam.cpu().numpy()
        # same kernels in the same order: equal to the tolerance of the line-smoother parity test
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    gpu.close()


def test_noalloc_line_smooth_rejects_meshes_beyond_its_scratch():
    from paper_2210_11797_gb300 import hmg
    w = I.cubed_sphere(48, 30)                    # 1,257,984 trace unknowns > 1,048,576
    gpu = hmg.Solver(w.hier, w.coeffs, tol=w.tol)
    b = torch.zeros(gpu.ntrace, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(b)
    L = hmg.lib()
    st = L.hmg_line_smooth_noalloc(gpu.ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(lam.data_ptr()), 1)
    assert st == 1 and b"1048576" in L.hmg_last_error(gpu.ctx)
    gpu.close()
