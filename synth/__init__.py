"""Seeded synthetic inputs for the spherical Poisson solver.

Shared by the tests, the benchmark and (as inputs only) the oracle.  The
module holds none of the solver's arithmetic: it samples real spherical
harmonic series on the longitude-colatitude grid and the closed-form
solutions of Poisson's equation for them (the Laplacian eigen-relation
Delta Y_l^m = -l(l+1) Y_l^m on the unit sphere).
"""

from .sh import (  # noqa: F401
    colatitudes,
    longitudes,
    random_sh_coeffs,
    single_sh_coeffs,
    synthesize,
    synthesize_many,
    batched_workload,
    poisson_exact,
    workload,
    WORKLOADS,
)
