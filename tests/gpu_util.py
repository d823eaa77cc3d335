"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the oracle."""

import numpy as np

# Gaps of the same run whose lines were grouped into blocks differently (a
# batch against single runs, the small-grid kernel against the persistent
# one, a mixed launch): the per-block partial sums are FP32 and only the sum
# across blocks is FP64, so such gaps agree to FP32 rounding of a block's sum.
GROUPING_RTOL = 1e-6


def cuda_available():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def gpu_gs(I, phi0, iters, grid=None, final_residual=True, aliased=False):
    """Run the CUDA path; returns numpy (phase, r, g) and the status code."""
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib

    build_lib.build()
    ny, nx = I.shape
    with GerchbergSaxton(nx, ny, final_residual=final_residual) as gs:
        if grid:
            gs.set_grid(grid)
        It = torch.from_numpy(np.ascontiguousarray(I, np.float32)).cuda()
        Pt = torch.from_numpy(np.ascontiguousarray(phi0, np.float32)).cuda()
        out, r, g = gs.run(It, Pt, iters, phase_out=Pt if aliased else None)
        st = gs.status()
        from paper_1302_0120_gb300 import _binding as B

        assert B.gs_check_workspace(gs.handle) == B.GS_OK  # no write past a workspace buffer
        return out.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy(), st


def aligned_rel_err(phi_gpu, u_ref):
    """min over a global phase alpha of ||exp(i phi_gpu) - e^{i alpha} u_ref|| / ||u_ref||.

    The iteration is equivariant under u -> e^{i alpha} u, so a global phase
    difference is not an error (it random-walks between implementations)."""
    ua = np.exp(1j * phi_gpu.astype(np.float64))
    c = np.vdot(ua, u_ref)  # sum conj(ua) u_ref
    ua = ua * np.exp(1j * np.angle(c))
    return float(np.linalg.norm(ua - u_ref) / np.linalg.norm(u_ref))
