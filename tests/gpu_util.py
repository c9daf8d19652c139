"""Helpers shared by the GPU tests: build one seeded problem on the device
through the C ABI and the same problem on the host through the oracle."""
import numpy as np

from paper_1508_01256_gb300 import inputs


def device_problem(ccs, p: inputs.Problem, device="cuda"):
    import torch
    csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed, device=device)
    x = torch.from_numpy(p.x).to(device)
    y = ccs.measure(ptr, cols, x, p.m, p.d)
    return csc, ptr, cols, y


def oracle_problem(orc, p: inputs.Problem):
    A = orc.make_expander(p.n, p.m, p.d, p.a_seed)
    y = orc.measure(A, p.m, p.x)
    return A, y


def upload_matrix(orc, A: np.ndarray, m: int, device="cuda"):
    """CSC + CSR of a host matrix (CSR from the oracle's transpose)."""
    import torch
    ptr, cols = orc.transpose(A, m)
    return (torch.from_numpy(np.ascontiguousarray(A)).to(device),
            torch.from_numpy(ptr).to(device), torch.from_numpy(cols).to(device))


def assert_same_decode(gpu, ref, check_hist=True):
    """Bitwise comparison of a device decode with the oracle's."""
    xg = gpu.x_hat.cpu().numpy()
    rg = gpu.r.cpu().numpy()
    assert gpu.status == ref["status"], (gpu.status, ref["status"])
    assert gpu.iterations == ref["iterations"], (gpu.iterations, ref["iterations"])
    assert gpu.r0_final == ref["r0_final"]
    assert np.array_equal(xg.view(np.int64), ref["x_hat"].view(np.int64)), \
        f"x_hat differs at {np.nonzero(xg.view(np.int64) != ref['x_hat'].view(np.int64))[0][:10]}"
    assert np.array_equal(rg.view(np.int64), ref["r"].view(np.int64)), \
        f"r differs at {np.nonzero(rg.view(np.int64) != ref['r'].view(np.int64))[0][:10]}"
    if check_hist and gpu.r0_hist is not None:
        assert list(gpu.r0_hist) == list(ref["r0_hist"])
