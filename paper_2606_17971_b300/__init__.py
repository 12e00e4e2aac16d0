"""B300-native (sm_103a) online spectral deflation for state-constrained
optimal control: the A-DEF2-deflated Jacobi-PCG inner solve of the primal
active-set loop, behind the C ABI declared in ``include/sdf.h``.

Importing the package is cheap; ``paper_2606_17971_b300.sdf`` loads the CUDA
library (and raises if it is missing).  ``paper_2606_17971_b300.workloads``
holds the seeded synthetic inputs.
"""

__all__ = ["sdf", "workloads"]
