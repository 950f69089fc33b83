"""Seeded synthetic inputs for the Wannier-interpolated linewidth path.

This package only draws numbers: lattices, real-space vector sets, Wannier-space
matrices H(Re), Phi(R), g(Re,Rp), k/q point lists and run parameters.  It holds
none of the method's arithmetic (no Fourier sums, no eigensolves, no self-energy
terms), so both the CPU oracle and the CUDA path can be fed from it without
sharing any computation.
"""
from .models import (  # noqa: F401
    WannierModel,
    Workload,
    LATTICES,
    lattice_shells,
    box_vectors,
    uniform_grid,
    random_points,
    make_model,
    make_workload,
    WORKLOADS,
    load_kpoint_file,
    tight_binding_model,
    diatomic_chain_model,
    einstein_model,
)
