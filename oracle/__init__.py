"""Oracle: a plain, slow, dense CPU FP64 implementation of the qHP TD-PMCHWT
marching-on-in-time scheme, written from the paper's equations.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import it. It shares no code with the CUDA
path; from the package it imports nothing but the seeded input generators
(paper_2510_07989_gb300.inputs: meshes, the operator assembler, quadrature
tables), which carry the MOT step's inputs and none of its arithmetic.

Route (different from the CUDA product form on purpose):
  * explicit incidence matrices Lambda, Sigma (Section IV-B);
  * dense projectors with Moore-Penrose pseudo-inverses (Section IV-B);
  * dense G^{-1}, explicit left factors T^{Sigma H} G^{-1}, T^Lambda G^{-1} P^{Lambda H};
  * explicit dense Q_k = Q_k^ll + Q_k^ls + Q_k^sl + Q_k^ss (Section V-B);
  * one LU factorisation of Q_0 and the MOT recursion Eq. (MOT).
"""
