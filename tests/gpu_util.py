"""Helpers of the GPU tests: run a workload through the C ABI and compare."""
import numpy as np

from paper_2502_06319_gb300 import cosmica as cz


def torch():
    import torch as t
    return t


def gpu_run(job, precision=cz.PREC_FP64, host_out=False, params=None, with_lw=False):
    """Propagate a workload with cosmica_propagate; returns (numpy dict, ExitBuffers, model)."""
    t = torch()
    m = cz.Model(cz.make_params(params or job.params, precision))
    sp = cz.make_species(job.species)
    out = cz.ExitBuffers(job.n_particles, device="cpu" if host_out else "cuda", pin_memory=host_out,
                         with_lw=with_lw)
    cz.cosmica_propagate(m.h, sp, job.T_in, job.n_per_energy, job.seed, out)
    t.cuda.synchronize()
    return out.numpy(), out, m


def gpu_spectrum(job, out):
    t = torch()
    nE, nb = len(job.T_in), job.bins.n
    J = t.empty(nE, dtype=t.float64, device="cuda")
    S = t.empty(nE, dtype=t.float64, device="cuda")
    H = t.empty(nE * (nb + 3), dtype=t.int64, device="cuda")
    cz.cosmica_spectrum(out, cz.make_species(job.species), job.T_in,
                        cz.make_bins(job.bins.P_min, job.bins.P_max, nb), J, S, H)
    t.cuda.synchronize()
    return H.cpu().numpy().view(np.uint64).reshape(nE, nb + 3), J.cpu().numpy(), S.cpu().numpy()


def compare_paths(g, o, rel=1e-10):
    """Fraction of paths with the same exit step and, among them, the worst relative state error."""
    same = (g["steps"] == o["steps"]) & (g["status"] == o["status"])
    worst = 0.0
    for k in ("r", "th", "ph", "lnP", "s"):
        a, b = g[k][same], o[k][same]
        if a.size:
            d = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
            if k == "ph":   # phi near 0 wraps; compare on the circle
                d = np.minimum(d, np.abs(np.abs(a - b) - 2 * np.pi) / np.maximum(np.abs(b), 1e-300))
            worst = max(worst, float(d.max()))
    return float(same.mean()), worst


def gpu_unbinned(job, out, formulation):
    t = torch()
    nE = len(job.T_in)
    J = t.empty(nE, dtype=t.float64, device="cuda")
    S = t.empty(nE, dtype=t.float64, device="cuda")
    cz.cosmica_spectrum_unbinned(out, cz.make_species(job.species), job.T_in, job.n_per_energy, formulation, J, S)
    t.cuda.synchronize()
    return J.cpu().numpy(), S.cpu().numpy()
