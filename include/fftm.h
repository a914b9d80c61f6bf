/*
 * fftm.h -- C ABI of the GB300 (sm_103a) hot path of the displacement-based
 * DTT/FFT fixed-point mechanical solver of arXiv 2607.05929 ("A robust and
 * versatile parallel FFT-based mechanical solver for general non-periodic and
 * periodic boundary conditions").
 *
 * One problem = one voxel grid on one GPU.  Per fixed-point iteration the
 * library runs, on the caller's CUDA stream (Algorithm 1, Sec. 2.4):
 *   finite-difference gradient -> constitutive law -> divergence and the
 *   equilibrium norms (Eqs. div_pol, equilibrium_condition) -> Anderson
 *   acceleration on p -> per-axis forward DCT/DST/DFT (Table 1) -> B0 or 2mu0
 *   discrete Green operator (Eqs. NSGO1_*, NSGO2_*) -> inverse transforms ->
 *   fluctuation displacement u^f.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an int status: 0 = OK, > 0 = a completed,
 *   non-fatal outcome (FFTM_NOT_CONVERGED), < 0 = an error.  Nothing throws
 *   across the ABI.  fftm_last_error() returns a thread-local text for the
 *   last error of the calling thread.
 * - Pointers are plain host or device pointers; the argument's name says
 *   which.  The library never keeps a caller pointer after a call returns:
 *   inputs are copied, outputs are written before the call returns (for
 *   device outputs: ordered on the problem's stream).
 * - Node fields are dense, component-major, x fastest:
 *   index = x + N1*(y + N2*(z + N3*q)), q = displacement component, with
 *   N_a = n_a + 1 nodes on a non-periodic axis and n_a on a periodic one
 *   (node n_a of a periodic axis is node 0; Sec. 2.1, Sec. 2.7.1).
 * - Voxel fields are dense, x fastest, point-major:
 *   index = x + n1*(y + n2*(z + n3*(c + nc*r))), r = voxel point (HEX1: one
 *   point; TETRA2: r = 0 tetrahedron T1, r = 1 tetrahedron T2), c = tensor
 *   component.  Gradients use G[i][q] = D_i u_q (c = 3 i + q); symmetric
 *   stresses use c = 0..5 for (11, 22, 33, 23, 13, 12).  A problem with a
 *   finite-strain law or FFTM_LAW_B0_LINEAR has non-symmetric stresses, stored
 *   with 9 components c = 3 i + q holding P_qi (P the first Piola-Kirchhoff
 *   stress, (div P)_q = d P_qi / d x_i).
 * - Field element type = the problem's precision (double for FFTM_FP64,
 *   float for FFTM_FP32).
 */
#ifndef FFTM_H
#define FFTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define FFTM_OK 0
#define FFTM_NOT_CONVERGED 1  /* max_iter reached; fields hold the last iterate */
#define FFTM_E_INVALID (-1)   /* bad argument or descriptor */
#define FFTM_E_NOMEM (-2)     /* device allocation failed or workspace too small */
#define FFTM_E_CUDA (-3)      /* a CUDA runtime call failed */
#define FFTM_E_DIVERGED (-4)  /* NaN / Inf in the equilibrium norms */
#define FFTM_E_UNSUPPORTED (-5)
#define FFTM_E_TIMEOUT (-6)   /* a bounded device-side wait gave up (a tensor-core pass
                                 whose MMA hand-over did not complete within about a
                                 second); the result of that call is undefined, the
                                 CUDA context stays usable */

/* ---- enumerations ----------------------------------------------------- */
enum fftm_bc { FFTM_BC_PERIODIC = 0, FFTM_BC_DIRICHLET = 1, FFTM_BC_NEUMANN = 2 };
enum fftm_scheme { FFTM_HEX1 = 0, FFTM_TETRA2 = 1 };
/* FFTM_GREEN_C0: the reference stiffness C0 : grad u = 2 mu0 grad u + lambda0 tr(grad u) 1
   (Sec. 2.6.1, Eq. TF_C0_behavior), whose discrete Green operator couples the three
   components at each frequency (Eq. FourierSGO_HEX1; TETRA2: Eqs. FourierSGO_TETRA2_1/2, a
   2 x 2 system per frequency).  Valid for normal-mixed BCs (Eq. SGO_BCs); this library builds
   it with every axis non-periodic, the same symmetry on both faces of an axis per component,
   and on each axis the normal component's symmetry opposite to the tangential ones' (normal
   Dirichlet and tangential Neumann, or the converse); FFTM_E_UNSUPPORTED otherwise. */
enum fftm_green { FFTM_GREEN_B0 = 0, FFTM_GREEN_MU0 = 1, FFTM_GREEN_C0 = 2 };
/* FFTM_FP32_TC: FP32 fields and residual (as FFTM_FP32), per-axis transforms
   as dense matrix contractions on the tensor cores (tcgen05) with BF16 operands
   and FP32 accumulation (transform lengths up to 288 node positions along x, the
   range's first node mod 4 included, and 352 along y and z; FFTM_E_UNSUPPORTED
   beyond). */
/* FFTM_FP32_TF32: FP32 fields and residual, per-axis transforms as dense matrix
   contractions on the tensor cores with TF32 operands (tcgen05 kind::tf32: the FP32
   fields and FP32 matrices are read as stored, the products carry 10-bit significands,
   FP32 accumulation), lengths up to 384 node positions per axis (FFTM_E_UNSUPPORTED
   beyond). */
enum fftm_precision { FFTM_FP64 = 0, FFTM_FP32 = 1, FFTM_FP32_TC = 2, FFTM_FP32_TF32 = 3 };

/* fftm_problem_desc.lambda0 / mu0: take the reference medium from the phases (Sec. 2.6, the
   paper's choice of half the sum of the extreme values of each Lame coefficient). */
#define FFTM_REF_AUTO (-1.0)
enum fftm_law {
  FFTM_LAW_ISO_ELASTIC = 0,   /* params: lambda, mu                          */
  FFTM_LAW_CUBIC_ELASTIC = 1, /* params: C11, C12, C44; quat = orientation     */
  FFTM_LAW_J2_LINHARD = 2,    /* params: lambda, mu, sigma_y, H: small-strain
                                 von Mises plasticity, linear isotropic hardening
                                 (yield stress sigma_y + H p), radial return from
                                 the committed state (Sec. 3.2); the state is
                                 committed when a load step converges           */
  FFTM_LAW_B0_LINEAR = 3,     /* params: lambda, mu: P = 2 mu G + lambda G.*I  */
  FFTM_LAW_SVK_CUBIC = 4,     /* finite strain, F = 1 + grad u: second Piola-
                                 Kirchhoff Pi = C : E, E = (F^T F - 1)/2, C cubic
                                 (params C11, C12, C44; quat), P = F Pi
                                 (Sec. 3.1.2)                                   */
  FFTM_LAW_NEO_HOOKE = 5,     /* finite strain, params mu, K: psi = mu/2 (J^(-2/3)
                                 tr(F^T F) - 3) + K/2 (J - 1)^2, P = F dpsi/dE
                                 (Appendix B)                                   */
  FFTM_LAW_CP_FCC = 6,        /* finite-strain FCC crystal plasticity (Sec. 3.4):
                                 F = F^e F^p, Pi = C : E^e (cubic C11, C12, C44,
                                 quat = lattice orientation), 12 {111}<110>
                                 systems, gdot_s = gdot0 |tau_s/tau_c|^n sign,
                                 Voce tau_c(Gamma) = tau0 + (tau_inf - tau0)
                                 (1 - exp(-h0 Gamma / (tau_inf - tau0))), one
                                 implicit increment of length dt per load step.
                                 params: C11, C12, C44, gdot0, n, tau0, tau_inf,
                                 h0, dt.  Not combinable with J2 phases.         */
  FFTM_LAW_LOG_J2 = 7         /* finite-strain perfect von Mises plasticity in the
                                 logarithmic strain space (Sec. 3.2, the porous
                                 medium): Hencky strain H = log(F^T F)/2 split
                                 additively into H^e + H^p, T = 2 mu dev H^e +
                                 K tr H^e 1 the stress conjugate to H (K = lambda
                                 + 2 mu / 3), yield sqrt(3/2) |dev T| = sigma0,
                                 backward-Euler radial return from the committed
                                 (H^p, p), second Piola-Kirchhoff S = T : d log C
                                 / d C (C = F^T F), P = F S.  params: lambda, mu,
                                 sigma0.  Committed when a load step converges.
                                 Not combinable with J2 or crystal-plasticity
                                 phases.                                        */
};

/* ---- descriptors ------------------------------------------------------ */
typedef struct fftm_material {
  int law;           /* enum fftm_law */
  double params[12]; /* law parameters, see enum fftm_law */
  double quat[4];    /* unit quaternion (w, x, y, z): crystal frame -> sample
                        frame; used by FFTM_LAW_CUBIC_ELASTIC */
} fftm_material;

typedef struct fftm_problem_desc {
  int n[3];                  /* voxels per axis, each >= 2 (Sec. 2.1)        */
  double h[3];               /* voxel sizes, > 0                             */
  const uint16_t* phase;     /* HOST pointer, n1*n2*n3 phase ids, x fastest;
                                copied, the caller keeps ownership           */
  int n_phases;              /* number of entries in materials, <= 65535      */
  const fftm_material* materials; /* HOST pointer, copied                    */
  int bc[3][2][3];           /* bc[axis][face][component], enum fftm_bc.
                                face 0 contains the origin.  A periodic axis
                                must be periodic on both faces, every comp.
                                Dirichlet -> u^f_q anti-symmetric, Neumann ->
                                symmetric (Eq. GeneralBCtobesolved).          */
  int scheme;                /* enum fftm_scheme (Sec. 2.5)                  */
  int green;                 /* enum fftm_green (Sec. 2.6.1 / 2.6.2 / 2.6.3) */
  double lambda0, mu0;       /* reference material; lambda0 ignored for MU0;
                                FFTM_REF_AUTO for either: half the sum of the
                                largest and smallest value over the phases
                                (fftm_host_reference_medium)                   */
  int precision;             /* enum fftm_precision                          */
  double tol;                /* equilibrium tolerance epsilon, > 0           */
  int max_iter;              /* I_max, >= 1                                  */
  int anderson_depth;        /* couples kept, 2..4 (0 disables Anderson)     */
  int anderson_period;       /* accelerate when m % period == period - 1     */
} fftm_problem_desc;

/* Prescribed displacement
     u*_q(x) = sum_a A[q][a] x_a + b[q] + sum_k Q[q][k] m_k(x),
     m = (x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2),
   x = physical node coordinates (node j of axis a at j*h_a).  u* supplies the
   Dirichlet values (Sec. 2.2); it must not depend on a periodic coordinate
   (FFTM_E_INVALID).  The quadratic terms carry bending and torsion loads (face
   rotations that grow along an axis); their discrete gradients are applied in
   closed form at the voxel points.

   Normal-mixed loading (Sec. 3.2, Eq. NMBC1: one component of <grad u*> imposed,
   the others adjusted at each iteration so that the mean stress vanishes in
   them): `mixed` is a bit mask over the symmetric strain components of u*
   (Voigt order 11, 22, 33, 23, 13, 12, bit k for the k-th).  After every
   residual the free components take the increment -(C0_FF)^-1 <sigma>_F, C0 the
   isotropic reference stiffness (lambda0, mu0), <sigma> the mean stress over the
   voxel points; the increment is added symmetrically to A, whose skew part and
   imposed components stay as given.  A's free entries are the first step's
   starting guess; a later step whose load has the same mask starts them from
   the values the previous mixed step ended with.  The step converges when err < tol
   and ||<sigma>_F|| / ||<sigma>|| < tol (tensor norms).  Requires small-strain
   laws (symmetric P) and non-periodic axes i and j for every free component ij
   (FFTM_E_INVALID otherwise).  0: A is imposed as given.  fftm_get_load returns
   the load with the adjusted A. */
typedef struct fftm_load {
  double A[3][3];
  double b[3];
  double Q[3][6];
  double T[3][2][3]; /* uniform Neumann tractions T[axis][face][component] (face 0 at
                        x_axis = 0, 1 at x_axis = L; outward normal convention,
                        traction_q = P_iq n_i; Sec. 2.2): the stress of the faces where
                        that component is Neumann, imposed through P* = 2 t at the
                        mirror voxel centres; non-zero only on such faces, else
                        FFTM_E_INVALID.  All zero: traction-free faces. */
  int mixed;  /* normal-mixed mask, 0 = none */
} fftm_load;

typedef struct fftm_step_report {
  int iterations;       /* Green applications performed (0 = initial guess converged) */
  int converged;        /* 1 if err < tol (a mixed load: and its mixed error)  */
  double err;           /* final equilibrium error (Eq. equilibrium_condition) */
  int n_accelerated;    /* Anderson steps taken                               */
  double mean_P[6];     /* volume mean of P over voxel points, (11,22,33,23,13,12) */
  double mean_G[9];     /* volume mean of the total gradient G[i][q]          */
} fftm_step_report;

typedef struct fftm_ctx fftm_ctx;
typedef struct fftm_problem fftm_problem;

/* ---- library ---------------------------------------------------------- */
const char* fftm_last_error(void);
int fftm_version(void);

/* Bind to CUDA device `device` (its primary context) and to `cuda_stream`
   (a cudaStream_t, or NULL for the legacy default stream).  All work of the
   problems created from this context is ordered on that stream. */
int fftm_ctx_create(fftm_ctx** out, int device, void* cuda_stream);
int fftm_ctx_destroy(fftm_ctx* ctx);

/* Device bytes a problem with this descriptor allocates to solve (fields, Anderson
   history, transform tables and matrices, law tables, internal variables, the staging
   buffer of host transfers, the device-decided step's history), an upper bound that
   includes the alignment of every allocation. */
int fftm_problem_workspace_bytes(const fftm_problem_desc* desc, size_t* bytes);

/* fftm_problem_create with every device allocation of the problem carved from a caller's
   device buffer (e.g. a torch tensor, so that the framework owns the memory): `workspace`
   (DEVICE pointer on the context's device, 256-byte aligned) of `bytes` >=
   fftm_problem_workspace_bytes(desc) (FFTM_E_NOMEM otherwise); the caller keeps ownership
   and must keep it alive until fftm_problem_destroy.  Allocations made after creation by
   optional features (fftm_set_load_field, fftm_set_face_traction, the test variant of
   FFTM_OP_RESIDUAL) are carved from what is left and return FFTM_E_NOMEM when it does not
   suffice, so pass more than the minimum when they are used. */
int fftm_problem_create_in(fftm_ctx* ctx, const fftm_problem_desc* desc, void* workspace, size_t bytes,
                           fftm_problem** out);

/* Validate the descriptor, derive per-component per-axis transform kinds and
   node ranges (Table 1; Sec. 2.7.2 "dismissed" points), build the frequency
   tables and law tables, allocate device memory (cudaMalloc; FFTM_E_NOMEM on
   failure), upload the phase map.  u^f starts at zero. */
int fftm_problem_create(fftm_ctx* ctx, const fftm_problem_desc* desc, fftm_problem** out);
int fftm_problem_destroy(fftm_problem* p);

/* Replace the phase map (HOST pointer, n1*n2*n3 ids < n_phases, copied). */
int fftm_set_phase(fftm_problem* p, const uint16_t* phase);

/* Set the prescribed displacement of the next load steps (Algorithm 1,
   "update the desired loading"). */
int fftm_set_load(fftm_problem* p, const fftm_load* load);

/* Non-uniform Neumann tractions on one face (Sec. 2.2; the uniform part is fftm_load.T, and
   the two add): t holds 3 x n_c x n_b values of the problem's precision, component-major,
   t[(q * n_c + c) * n_b + b] at the centre of face voxel (b, c), where b < c are the two
   in-plane axes (axis 0: (y, z); axis 1: (x, z); axis 2: (x, y)); outward normal convention
   (traction_q = P_iq n_i).  Imposed through P* = 2 t at the mirror voxel centres across the
   face (ghost voxels beyond the face's edges take the value of the face voxel they mirror).
   t is a HOST (t_is_device = 0) or device pointer, copied before the call returns; bytes must
   be 3 n_b n_c times the element size.  A component that is not Neumann on that face must be
   zero (FFTM_E_INVALID); so must the call for a periodic axis.  t = NULL removes the field.
   Takes effect at the next load step (or residual). */
int fftm_set_face_traction(fftm_problem* p, int axis, int face, const void* t, int t_is_device, size_t bytes);

/* A prescribed displacement given as a node field (Sec. 2.2: u* is any field carrying the
   Dirichlet values), added to the closed-form u* of fftm_set_load: 3 components in the dense
   node layout of the file header (problem precision), HOST (is_device = 0) or device pointer,
   copied before the call returns; bytes must be 3 N1 N2 N3 times the element size.  Its
   gradient at the voxel points is the scheme's stencil on its node values (Eqs. D1HG-D3HG,
   D1T1T2G-D3T1T2G); on a periodic axis the stored nodes make it periodic.  Its values at the
   Dirichlet nodes are the displacement imposed there (u^f vanishes at them).  NULL removes it.
   Not combinable with a normal-mixed load (FFTM_E_INVALID).  Takes effect at the next load
   step; a J2 problem's incremental residual takes its change since the last commit. */
int fftm_set_load_field(fftm_problem* p, const void* ustar, int is_device, size_t bytes);

/* The current load (HOST out): as set, with the free components of a mixed load
   at their latest adjusted values. */
int fftm_get_load(const fftm_problem* p, fftm_load* out);

/* Run Algorithm 1 for one load step from the current u^f (the previous
   step's converged field, zero initially).  When the step converges, the
   internal variables of J2 phases are committed from the converged field (a
   step that does not converge commits nothing).  Blocks until the report is
   written.  Returns FFTM_OK, FFTM_NOT_CONVERGED, or an error.  `err_history`
   (HOST, may be NULL) receives up to `history_len` per-iteration errors;
   `accel_history` (HOST, may be NULL) receives 1/0 per iteration for an
   Anderson step taken at that iteration. */
int fftm_solve_step(fftm_problem* p, fftm_step_report* report, double* err_history,
                    int* accel_history, int history_len);

/* ---- fields ----------------------------------------------------------- */
enum fftm_field {
  FFTM_FIELD_U = 0,      /* u^f, node field (3 comps; FP32: the high part)       */
  FFTM_FIELD_WORK = 1,   /* the p / spectral work field, node layout (3 comps)   */
  FFTM_FIELD_GRAD = 2,   /* total gradient G at voxel points (9 comps)           */
  FFTM_FIELD_STRESS = 3, /* stress at voxel points (6 comps, or 9 for problems
                            with non-symmetric stresses, see the layout above)  */
  FFTM_FIELD_D = 4,      /* residual D = div P at the nodes (3 comps), dismissed
                            node components 0; written by FFTM_OP_RESIDUAL       */
  FFTM_FIELD_STATE = 5,  /* committed internal variables at voxel points: J2
                            problems 7 comps (eps^p 11, 22, 33, 23, 13, 12 and
                            the cumulated plastic strain p), crystal plasticity
                            10 comps (F^p row-major, cumulated slip Gamma),
                            logarithmic J2 7 comps (H^p 11, 22, 33, 23, 13, 12
                            and p); zero in voxels of other laws; FFTM_E_INVALID for
                            problems without such a phase                    */
  FFTM_FIELD_U_LO = 6    /* FP32 problems carry u^f as an unevaluated sum hi + lo of
                            two floats: FFTM_FIELD_U reads and writes the high part,
                            this the low part (read only; FFTM_FIELD_U's write sets
                            it to zero); zeros for FP64 problems; node layout      */
};

/* Bytes of a field (dense layout above, problem precision). */
int fftm_field_bytes(const fftm_problem* p, int field, size_t* bytes);

/* Options of a problem (fftm_set_option):
   FFTM_OPT_RESIDUAL_PASSES  how the solver evaluates the residual (rows a1-a4) of problems
                             whose laws are all small-strain elastic: 1 = one pass over the
                             grid (gradient, law and divergence fused, the voxel-point stresses
                             kept on chip), 2 = two passes (stresses stored, then the
                             divergence), 0 (default) = whichever the library measured faster
                             for this grid shape on this GPU (timed once per shape and process;
                             fftm_tuning_table lists the choices).  Both forms give the same D;
                             problems with other laws always take two passes.
   FFTM_OPT_CUDA_GRAPH       1: a device-decided step (FFTM_OPT_DEVICE_LOOP 1, no normal-mixed
                             load, profiling off) captures its iterations into two CUDA graphs
                             per load step (the first lcm(5, anderson_period) iterations and the
                             next as many, which repeat) and replays the second until the
                             convergence flag is set, one host wait per replay; results are
                             bit-identical to 0 (the default: iterations enqueued one by one).
                             Launch counts then include the kernels replayed past the stop,
                             which return at once.  A stream that cannot be captured falls back
                             to 0.
   FFTM_OPT_RESIDUAL_TILE    the one-pass form's voxel tile height: 8 or 16 rows of 32
                             voxels per thread block, or 0 (default) = measured, as above.
   FFTM_OPT_DEVICE_LOOP      1 (default): the convergence test of each iteration (Eq.
                             equilibrium_condition against tol, the iteration limit, non-finite
                             norms) runs on the device; the host enqueues the iterations in
                             chunks of four and waits once per chunk, and the launches of a chunk
                             that follow the iteration that stopped the step do nothing.  0: the
                             host reads the norms after every residual.  Loads with a
                             normal-mixed part always take the host path (their free strain
                             components are updated on the host).  Both give the same iterates. */
enum fftm_option {
  FFTM_OPT_RESIDUAL_PASSES = 0,
  FFTM_OPT_RESIDUAL_TILE = 1,
  FFTM_OPT_DEVICE_LOOP = 2,
  FFTM_OPT_CUDA_GRAPH = 3
};
int fftm_set_option(fftm_problem* p, int option, int value);

/* Measured fused multiply-add throughput of a device (FLOP/s, an FMA counting two), in FP64
   (fp64 = 1) or FP32 (fp64 = 0): eight independent FMA chains per thread over all SMs, the best
   of three timed launches.  The denominator of an arithmetic-bound roofline (the FP64 path on
   this GPU is bound by its FP64 rate, a small fraction of the FP32 one). */
int fftm_device_fma_rate(int device, int fp64, double* flops_per_s);

/* The launch-shape choices the library has measured in this process, one line per shape
   ("key: choice (times)").  buf (HOST, may be NULL) receives up to len - 1 characters and a
   terminating 0; *needed (may be NULL) the size the whole table needs. */
int fftm_tuning_table(char* buf, size_t len, size_t* needed);

/* Node dimensions N[3] of the problem's node fields (N_a = n_a + 1 on a non-periodic
   axis, n_a on a periodic one; Sec. 2.1), its precision (enum fftm_precision) and its
   CUDA device, so a caller can size, type and place the device buffers it passes to the
   library.  HOST outputs; each may be NULL. */
int fftm_problem_layout(const fftm_problem* p, int N[3], int* precision, int* device);

/* Copy a field out.  dst is a device pointer if dst_is_device, else host.
   bytes must equal fftm_field_bytes().  GRAD and STRESS are evaluated from
   the current u^f on demand. */
int fftm_get_field(fftm_problem* p, int field, void* dst, int dst_is_device, size_t bytes);

/* Copy a field in (FFTM_FIELD_U, FFTM_FIELD_WORK or FFTM_FIELD_STATE).
   Values at dismissed node components are ignored and stored as zero; STATE
   is stored as given (a restart from a saved state). */
int fftm_set_field(fftm_problem* p, int field, const void* src, int src_is_device, size_t bytes);

/* ---- single steps of one iteration (each a row of the hot path) -------- */
enum fftm_op {
  FFTM_OP_RESIDUAL = 0,     /* u^f -> WORK = p (Eq. div_pol), D, and norms:
                               norms[0] = S_D, norms[1] = S_P, norms[2] = err.
                               With FFTM_OPT_RESIDUAL_PASSES 1 and a tile height
                               set, D and the norms come from the solver's
                               one-pass kernels (u^f as hi + lo) and WORK is
                               left as it was                                   */
  FFTM_OP_DT_FORWARD = 1,   /* WORK -> WORK, 3D forward DT (x, y, z; Table 1);
                               DCT/DST coefficient k of an axis sits at node
                               position lo + k; a periodic axis is stored in
                               halfcomplex order (real part of frequency k at
                               k, imaginary part at n - k)                      */
  FFTM_OP_GREEN = 2,        /* WORK -> WORK, multiply by the Green factor
                               -1 / (2 mu0 ||xi||^2 + lambda0 |xi_q|^2)
                               (0 where the denominator is null)               */
  FFTM_OP_DT_INVERSE = 3,   /* WORK -> WORK, 3D inverse DT, normalised          */
  FFTM_OP_GREEN_UPDATE = 4  /* WORK (p) -> u^f: forward DT, Green, inverse DT,
                               with the z pass fused (the solver's path)        */
};

/* Run one step on the problem's stream; `norms` (HOST, 3 doubles) is
   written for FFTM_OP_RESIDUAL and may be NULL otherwise.  Blocks until done. */
int fftm_apply(fftm_problem* p, int op, double* norms);

/* Number of kernels the library launched on this problem since creation. */
int fftm_kernel_launches(const fftm_problem* p, long long* count);

/* Zero u^f, the acceleration history and the J2 state (a fresh load sequence). */
int fftm_reset_state(fftm_problem* p);

/* Per-kernel timing with CUDA events on the problem's stream (off by default).
   While enabled, every launch of the solver is bracketed by two events; the
   elapsed times are accumulated per category when the stream is next
   synchronised by the library.  Categories (FFTM_KCAT_*): */
enum fftm_kcat {
  FFTM_KCAT_RESIDUAL = 0,  /* gradient + law + divergence + norm reduction      */
  FFTM_KCAT_PASS_X = 1,    /* x-axis transform passes (forward and inverse)      */
  FFTM_KCAT_PASS_Y = 2,    /* y-axis transform passes                            */
  FFTM_KCAT_PASS_Z = 3,    /* fused z forward + Green + z inverse                */
  FFTM_KCAT_ANDERSON = 4,  /* Gram, least squares, combination                   */
  FFTM_KCAT_OTHER = 5,     /* statistics, packing, standalone steps              */
  FFTM_KCAT_COUNT = 6
};
int fftm_set_profiling(fftm_problem* p, int enable);
/* ms[c] = total milliseconds, launches[c] = launches of category c since the
   last fftm_set_profiling(p, 1); both HOST arrays of n >= FFTM_KCAT_COUNT. */
int fftm_kernel_times(const fftm_problem* p, double* ms, long long* launches, int n);

/* ---- residual evaluation without allocation ---------------------------------
   No counterpart in the paper: an interface for callers that may not allocate
   device memory where they need a residual -- code running while a CUDA stream
   is captured into a graph (a cudaMalloc there breaks the capture), frameworks
   whose caching allocator or memory pool must own every device byte, and
   fixed-memory real-time loops.

   Evaluates D = div P (+ D*) and the norms of a caller-supplied u^f exactly as
   FFTM_OP_RESIDUAL does (same kernel), on the problem's stream, without any
   cudaMalloc/cudaFree:
     u_dev      DEVICE, input, the dense node layout of FFTM_FIELD_U in the
                problem's precision (FP32 problems read the field as plain floats)
     D_dev      DEVICE, output, same layout; dismissed node components get 0
     norms_dev  DEVICE, output, 3 doubles: S_D, S_P, err
   Asynchronous: results are ready when the problem's stream reaches them.
   Scratch: the reduction's block partials live in a file-scope device array
   of 16384 doubles (128 KiB) that every GPU loading the library holds until
   the process exits (the residual kernels use at most 2432 blocks, 2 slots
   each; a launch needing more than 16380 slots would be rejected with
   FFTM_E_UNSUPPORTED and a message); the voxel-point stresses go to a buffer
   the problem allocated when it was created.  Every slot read is written earlier in the same call, so nothing
   needs clearing; all calls share the array, so calls that overlap on the GPU
   (other streams, other threads, other problems on the same device) race.
   The first call on a device looks the array's device address up
   (cudaGetSymbolAddress): make that first call before any stream capture. */
int fftm_residual_noalloc(fftm_problem* p, const void* u_dev, void* D_dev, double* norms_dev);

/* ---- host-only utilities (no device work; callable without a GPU) -------- */

/* 1D transform kinds of Table 1 (the kind a component takes along an axis from its
   pair of face conditions: periodic -> DFT, N/N -> DCT-I, N/D -> DCT-III, D/D ->
   DST-I, D/N -> DST-III). */
enum fftm_dt_kind { FFTM_DT_DFT = 0, FFTM_DT_DCT1 = 1, FFTM_DT_DCT3 = 2, FFTM_DT_DST1 = 3, FFTM_DT_DST3 = 4 };

/* The dense matrix of a 1D transform (Table 1) or of its inverse, as the tensor-core
   path applies it: L x L over the kind's node range (L = n + 1, n, n - 1 for DCT-I,
   DFT/DCT-III/DST-III, DST-I), row-major, out[k L + c] = weight of node lo + c in
   output k; the DFT in halfcomplex order (row k <= n/2: the cosine sum, row n - k:
   minus the sine sum).  n voxels, 2 <= n <= 4096; inverse 0 or 1.  out (HOST, L*L
   doubles) may be NULL to query L; *L_out receives L.  FFTM_E_INVALID on a bad
   argument. */
int fftm_host_dense_transform(int kind, int n, int inverse, double* out, int* L_out);

/* Test export: the 1D transform of Table 1 of `kind` over an axis of n voxels (inverse 1:
   its normalised inverse), computed on GPU `device` by the library's FP64 transform pass
   (the kernels FFTM_OP_DT_FORWARD and FFTM_OP_DT_INVERSE run): a temporary problem of
   n x 2 x 2 voxels, periodic along y and z, carries the data as a constant along them.
   in, out: HOST arrays of L doubles (L as for fftm_host_dense_transform), node position
   lo + c of the kind's range at index c, the coefficients in the library's storage (DCT/DST
   coefficient k at k, the DFT in halfcomplex order).  The 3D form is FFTM_OP_DT_FORWARD on
   a problem's WORK field.  FFTM_E_INVALID on a bad argument; the errors of problem creation
   otherwise. */
int fftm_dt1d(int device, int kind, int n, int inverse, const double* in, double* out);

/* The reference medium a descriptor asks for: lambda0 and mu0 as given, or, for the one set to
   FFTM_REF_AUTO, (max + min) / 2 over the phases of their Lame pair: lambda, mu for the
   isotropic, J2, B0-linear and logarithmic J2 laws; lambda = C12, mu = (C44 + (C11 - C12) / 2)
   / 2 for the cubic ones (elastic, St-Venant-Kirchhoff, crystal plasticity); lambda = K -
   2 mu / 3 for Neo-Hooke.  d: HOST pointer; FFTM_E_INVALID on NULL arguments or an AUTO value
   without materials.  fftm_problem_create applies it before validating the descriptor. */
int fftm_host_reference_medium(const fftm_problem_desc* d, double* lambda0, double* mu0);

/* The normal-mixed strain increment (see fftm_load.mixed): d = -(C0_FF)^-1 <sigma>_F on
   the free components of `mask`, zero elsewhere, C0 the isotropic reference stiffness
   (lambda0, mu0 > 0).  sig and d_out: HOST 3x3 row-major. */
int fftm_host_mixed_increment(const double* sig, int mask, double lambda0, double mu0, double* d_out);

/* The logarithmic J2 law (FFTM_LAW_LOG_J2) at one voxel point, evaluated on the host by the
   same code the kernels run (FP64): G (9, G[3 i + q] = D_i u_q), params (lambda, mu, sigma0),
   st (7: the committed H^p 11, 22, 33, 23, 13, 12 and p) -> S (9, S[3 i + q] = P_qi) and, when
   st_out is not NULL, the returned state (7).  All HOST pointers; FFTM_E_INVALID on NULL. */
int fftm_host_log_j2(const double* G, const double* params, const double* st, double* S, double* st_out);

#ifdef __cplusplus
}
#endif
#endif /* FFTM_H */
