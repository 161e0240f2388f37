"""Shared helpers of the GPU tests: run the CUDA path, compare with the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def sgf():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1603_03142_gb300 import sgf as mod
    return mod


def run_gpu(plan, sigma):
    """Device solve of numpy sigma levels; returns numpy float64 (fx, fy) lists."""
    dt = torch.float64 if plan.precision == 0 else torch.float32  # FP32 and BF16X take float
    sig = [torch.from_numpy(np.ascontiguousarray(s)).to(device="cuda", dtype=dt) for s in sigma]
    fx, fy = plan.solve(sig)
    torch.cuda.synchronize()
    return [t.double().cpu().numpy() for t in fx], [t.double().cpu().numpy() for t in fy]


def rel_linf_levels(nest, gx, gy, ox, oy):
    """Per level: max over uncovered cells and both components of |F - F_oracle| / max |F_oracle|."""
    out = []
    for l in range(nest.levels):
        keep = ~nest.covered_mask(l)
        scale = max(np.abs(ox[l][keep]).max(), np.abs(oy[l][keep]).max())
        err = max(np.abs(gx[l] - ox[l])[keep].max(), np.abs(gy[l] - oy[l])[keep].max())
        out.append(err / scale)
    return out


def tol(precision: str, n: int) -> float:
    """Parity bound, relative L-infinity against the FP64 oracle.

    fp32: 1e-5, the bound the method is held to.  fp64: 1e-12 up to the size
    where table roundoff reaches it, then 0.2 eps n^2.  Both sides evaluate the
    same closed forms whose double differences cancel: corner antiderivatives
    grow like n (lattice units) while the differences shrink like 1/distance^2,
    so every table entry carries ~eps n absolute error, and a force sums n^2 of
    them weighted by densities of either sign: ~eps n^2 relative to a force of
    order one.  Measured on the tapered lognormal grid (the worst of the
    workloads): 9.2e-14 (n = 64), 3.0e-13 (128), 1.0e-12 (256), 5.1e-12 (512),
    1.9e-11 (1024), 6.9e-11 (2048), i.e. 0.07-0.1 eps n^2.  bf16x: 1e-4, the
    bound of the split-BF16 tensor-core path (each radix-16 DFT keeps about 16
    significant bits of its operands)."""
    if precision == "bf16x":
        return 1e-4
    if precision == "fp32":
        return 1e-5
    return max(1e-12, 0.2 * float(np.finfo(np.float64).eps) * n * n)
