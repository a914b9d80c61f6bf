"""FP64 CPU oracle for the per-iteration hot path of the DTT/FFT displacement solver.

TEST INFRASTRUCTURE.  This package is a plain, slow, obviously-correct
restatement of the paper's method (arXiv 2607.05929, "A robust and versatile
parallel FFT-based mechanical solver for general non-periodic and periodic
boundary conditions") in NumPy/SciPy, in FP64.  It shares no code with the
CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path never does.

Modules and what they restate:

* ``bc``          BC -> symmetry -> per-axis transform kind (Sec. 2.2, Eq. GeneralBCtobesolved; Table 1)
* ``transforms``  the five forward DTs of Table 1 and their inverses (Sec. 2.4, Sec. 2.7.2)
* ``stencils``    HEX1 / TETRA2 gradient and divergence with ghost voxels (Sec. 2.5, Remark 1)
* ``green``       B0 and 2mu0 discrete Green operators (Sec. 2.6.2-2.6.3, Eqs. NSGO1_*, NSGO2_*)
* ``laws``        small-strain constitutive laws (Sec. 3.1; cubic elasticity as in Sec. 3.3; J2, Sec. 3.2)
* ``finite``      finite-strain laws: St-Venant-Kirchhoff, Neo-Hookean (Appendix B), FCC crystal
                  plasticity (Sec. 3.4), logarithmic J2 (Sec. 3.2)
* ``mixed``       normal-mixed loading (Eq. NMBC1)
* ``anderson``    Anderson acceleration on p (Sec. 2.3, Algorithm 1)
* ``solver``      Algorithm 1, one load step (with Neumann tractions through ``stencils``)
* ``direct``      the same discrete problem assembled as a sparse matrix and solved directly

Parity status of each part is stated in the module headers.  Anderson's
combination is pinned by identities of affine maps (the mix of dim + 1 couples
lands on the fixed point, its residual is M r_min, a 3-free-DOF solve reaches
the solution right after its first mix); the accelerated iterates of a general
problem have no closed form (parity unpinned beyond self-consistency: the skip
decisions are fixed by the stated rule, and the fixed point reached is pinned
by the direct solve and the laminate closed forms).  The crystal-plasticity law is pinned by its
single-slip recursion and the full-field solve by a two-crystal laminate past yield
(traction continuity solved independently); its full-field polycrystal response is
parity unpinned beyond that (no closed form).
"""
