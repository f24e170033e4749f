"""B300-native Yee-Maxwell + LLG solver (arxiv 2510.22221, section "Numerical
Model"): a C-ABI CUDA library (include/fdtd_llg.h, built for sm_103a) with a
thin Python binding.  There is no CPU fallback: without the CUDA library or a
GPU every entry point raises."""
from ._abi import LLGError, load as load_library
from .solver import FdtdLlg, Material
from .spectra import fit_coupling, fit_modes

__all__ = ["FdtdLlg", "Material", "LLGError", "load_library", "from_workload", "configure", "fit_modes",
           "fit_coupling"]


def from_workload(w, probe_capacity=None, energy=True, llg_fixed_iter=0, llg_tol=1e-6, llg_max_iter=20,
                  torch_memory=True):
    """Create and configure a solver for a ``workloads.Workload``."""
    sim = FdtdLlg.create(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, courant_factor=w.courant, llg_tol=llg_tol,
                         llg_max_iter=llg_max_iter, llg_fixed_iter=llg_fixed_iter,
                         probe_capacity=probe_capacity or max(w.steps, 1), energy=energy, torch_memory=torch_memory)
    configure(sim, w)
    return sim


def configure(sim, w):
    """Materials, sources and probes of a ``workloads.Workload`` onto an instance."""
    table = [Material(**m) for m in w.materials]
    sim.set_materials(w.mat_id, table, w.hbias, w.eps_design, w.design_box)
    for s in w.sources:
        sim.set_source(s["comp"], s["i"], s["j"], s["k"], s["J0"], s["f0"], s["Tp"], s["tpk"])
    for p in w.probes:
        sim.add_probe(*p)
    if getattr(w, "pml", None):
        q = w.pml
        sim.set_pml(q["layers"], q["order"], q["scale"], q["kappa_max"], q["alpha_max"])
    return sim
