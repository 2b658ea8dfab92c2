"""CPU oracle for the Leja-point exponential-integrator hot path.

ORACLE — test infrastructure only.  Plain, slow, obviously correct FP64 code
(numpy, with Python `decimal` for the divided differences).  Only `tests/`,
`__graft_entry__.smoke()` and `bench.py`'s CPU-baseline / reference legs may
import it.  It shares no code with the CUDA library and imports nothing from
the `paper_1309_4616_gb300` package.

Modules
  leja       Leja points on [-2, 2], scalar phi_k, divided differences,
             the a-priori substep schedule (Sec. II-C, Eq. (3)).
  operators  Row assembly of the stencil operators and the CSR graph operator,
             Gershgorin interval (Sec. III-A, III-B).
  newton     The Newton-form Leja iteration, phi_k(hA)v with substeps,
             exponential Euler (Eq. (2)) and exponential Rosenbrock-Euler;
             the fixed-count form and the no-restart driver.
  mlp        The schedule network: forward, loss, backward, Adam (FP64).
  learned    Features, decision rule and phi_1 under the learned schedule,
             with the plain method as fallback.
  dense      phi_k(hA)v by definition: expm of an augmented matrix.
  skew       phi_k(-i h H)v for a real symmetric H (complex products, K = C):
             complex divided differences at the real Leja points.
  closed     Closed forms: sine / cosine eigenbases of constant-coefficient
             operators, the analytic Gaussian.
"""
