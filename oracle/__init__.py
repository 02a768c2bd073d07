"""FP64 CPU oracle of the finite element discrete Boltzmann method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (separate velocity-set, mesh, operator
and residual construction); the only module both sides read is the seeded
input generator ``paper_2012_13487_gb300.inputs``, which holds none of the
method's arithmetic.

Everything here is plain NumPy in float64, written step by step from
Ganeshan & Williams, "A finite element discrete Boltzmann method for high
Knudsen number flows" (arXiv 2012.13487):

* ``velset``  -- Gauss-Hermite and Newton-Cotes velocity sets (Sec. II.A.3,
  Table 1).
* ``mesh``    -- structured split-square triangulation, unstructured
  triangulations given as vertex / triangle lists, and their face
  connectivity (Sec. II.B.1, Sec. III).
* ``ops``     -- nodal DG operators on the reference triangle
  (Sec. II.B.1, eq. byparts), built from a Legendre-product basis and
  collapsed-coordinate quadrature.
* ``dg``      -- moments, Hermite equilibrium (eq. feq), diffuse walls
  (eq. FullBC / UsedBC), the strong-form DG residual equivalent to
  eq. byparts, LSRK(5,4) time marching, diagnostics.
* ``couette`` -- the linearized Couette closed form (eq. exact, repaired)
  and a discrete-velocity steady solve that checks it.
* ``implicit`` -- SDIRK time marching (backward Euler and two fourth-order
  tableaux, Sec. II.B.3) with Newton's method on a dense finite-difference
  Jacobian.

Parity status of each function is stated in its docstring; the cavity
workload has no printed solution, so beyond the method invariants its
parity is "parity unpinned" (oracle <-> GPU agreement only).
"""
