"""CPU oracle for the heterogeneous-DSA S_N transport path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 restatement of
what the paper's method computes (upwind DG S_N sweep, source iteration, diffusion
synthetic acceleration restricted to the thick subdomain, and the adjoint used for
gradients).  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does, and it shares no code with
the CUDA library.  It reads its inputs from the seeded generators in
paper_2001_09196_gb300.inputs, which hold none of the method's arithmetic.

Every function cites the passage it follows.  Readings of passages that are silent,
ambiguous or garbled are stated where they are used.
"""
from .quadrature import level_symmetric, level_symmetric_octant  # noqa: F401
from .transport import Transport, CycleError  # noqa: F401
