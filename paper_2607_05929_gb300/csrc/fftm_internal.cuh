// Internal types of the fftm library: transform plans, kernel parameter
// blocks and the launchers each .cu file provides.  Not part of the ABI.
#pragma once

#include <cuda.h>  // CUtensorMap (the TMA descriptor type; no driver call is made through it here)
#include <cuda_runtime.h>
#include <stdint.h>

namespace fftm {

// One-dimensional transform kinds, one per pair of face symmetries of a node
// field (Table 1): P/P -> DFT, S/S -> DCT-I, S/A -> DCT-III, A/A -> DST-I,
// A/S -> DST-III.
enum Kind { K_DFT = 0, K_DCT1 = 1, K_DCT3 = 2, K_DST1 = 3, K_DST3 = 4 };

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

constexpr int MAX_STAGES = 16;

// Plan of the 1D transform of one displacement component along one axis.
// Every DT is evaluated through one complex FFT of length M (M = n for the
// DFT, 2n for the DCT/DST kinds), two real pencils packed per complex pencil.
template <typename T>
struct AxisPlan {
  int kind;
  int n;      // voxels along the axis
  int lo, L;  // node range of the transform (positions lo .. lo + L - 1)
  int M;      // complex FFT length
  int nst;    // number of FFT stages
  int radix[MAX_STAGES];
  const int16_t* perm;               // M: input position of sequence index m
  const typename V2<T>::t* tw;       // M: exp(-2 pi i t / M)
  const typename V2<T>::t* qw;       // n + 1: exp(i pi j / (2 n))
};

// One axis pass over the three components of a node field.
template <typename T>
struct PassParams {
  const T* in[3];
  T* out[3];
  // optional accumulation at store (last inverse pass of the solver update):
  // out = base + scale * value, as an unevaluated hi + lo pair when out_lo is set
  const T* base[3];
  const T* base_lo[3];
  T* out_lo[3];
  int axis;
  int N[3];             // node dims
  long long stride[3];  // element strides of x, y, z
  AxisPlan<T> plan[3];
  int inverse;
  T scale[3];
  // fused forward z -> Green -> inverse z (axis 2 only)
  int fused;
  const T* S2[3][3];  // [q][axis] sin^2(xi/2) by frequency index
  const T* C2[3][3];  // [q][axis] cos^2(xi/2)
  int flo[3][3];      // [q][axis] node position of frequency index 0
  int fL[3][3];       // [q][axis] number of frequencies
  T hf[3];            // 4 / h_a^2
  T two_mu0, lam0;
  int tetra;
  T gscale[3];        // inverse-transform normalisation folded into the Green factor
  const int* stop;    // device flag: nonzero once the load step has stopped (the launch does nothing)
};

// Stencil + law + divergence (one fixed-point residual evaluation).
template <typename T>
struct ResParams {
  const T* u[3];    // u^f (high part in FP32)
  const T* ulo[3];  // low part of u^f (FP32 only; null otherwise)
  T* D[3];          // D = div P at the nodes (dismissed components 0)
  T* p[3];          // p = div(R0 : grad u^f) - D (test variant only)
  const uint16_t* phase;
  const int* law_id;  // per phase
  const T* law_c;     // per phase, LAWC coefficients
  const T* law_m;     // per phase, the elastic Mandel stiffness as 9 (2 x 2) blocks (36 entries)
  int n[3], N[3];
  int periodic[3];
  long long sy, sz;  // node strides (x stride 1)
  long long vy, vz;  // voxel strides
  T Gs[9];           // uniform gradient of the affine part of u*
  int quad;          // 1 if u* has quadratic terms
  // u* given as a node field (fftm_set_load_field, the problem's node layout nsy / nsz), added
  // to the closed-form part; us_n: the field at the last commit (J2 increments), or null
  const T* us[3];
  const T* us_n[3];
  T Qc[3][6];        // their coefficients: x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2
  T hh[3];           // voxel sizes
  // J2 phases are evaluated incrementally from the last commit: the state holds the
  // elastic strain e_n (11,22,33,23,13,12) and p_n per voxel point [r][7][voxel], and
  // the trial strain is e_n + sym(grad(u^f - u^f_n) + grad(u* - u*_n)).
  T* state;          // null: no phase with internal variables
  int nst;           // state components per voxel point: 7 (J2, logarithmic J2) or 10 (crystal plasticity)
  int slaw;          // the law with internal variables: 1 J2, 2 crystal plasticity, 4 logarithmic J2, 0 none
  int c0;            // the reference stiffness of tau is C0 (lambda0 tr(G) 1) instead of B0 (lambda0 G_ii)
  const T* un[3];    // u^f at the last commit (high part in FP32)
  long long nsy, nsz;  // node strides of un (the problem's layout; sy, sz may describe a caller's)
  const T* unlo[3];  // its low part (FP32 only)
  T dGs[9];          // gradient of the affine part of u* - u*_n
  int dquad;         // 1 if the quadratic part of u* - u*_n is non-zero
  T dQ[3][6];        // its coefficients
  // Incremental residual (J2 problems after their first commit): k_stress stores the
  // stress increment P - P_n and k_div adds D_n = div P_n, the residual at the commit,
  // so that FP32 rounding scales with the increment instead of the stress.
  int inc;
  const T* Dn[3];
  T lam0, two_mu0;
  T wdiv[3];         // 1 / (4 h_i)
  T wgrad[3];        // HEX1: 1 / (4 h_i); TETRA2: 1 / (2 h_i)
  int sgn[3][3][2];  // [q][axis][face] +1 symmetric (Neumann), -1 anti-symmetric (Dirichlet)
  int lo[3][3], hi[3][3];  // [q][axis] transformed node range
  // Uniform Neumann tractions tr[axis][face][q] (outward normal convention); at the nodes of
  // a loaded face the divergence reads the imposed stress P*_aq = 2 (-1)^(face+1) tr at the
  // ghost voxels across it (incremental form: the traction change since the commit)
  int traction;
  T tr[3][2][3];
  // Non-uniform tractions per face (null: none): tface[a][f][q * nb * nc + vb + nb * vc] over
  // the face's voxel centres (b < c the in-plane axes); the incremental form subtracts the
  // committed field tface_n
  const T* tface[3][2];
  const T* tface_n[3][2];
  T* vs;             // voxel-point stress buffer [r][c][voxel] (c < NC, see fftm_stencil.cuh)
  int sym;           // 1: every law gives a symmetric P (6 stored components)
  int two_pass;      // 1: evaluate the residual as two grid passes even where one pass serves
  int fused_fy;      // voxel tile height of the one-pass residual (8 or 16)
  double* partial;   // per block: S_D, S_P
  const int* stop;   // device flag: nonzero once the load step has stopped (the launch does nothing)
};

constexpr int LAWC = 40;

// Dynamic shared memory opt-in of the axis-pass kernels: one value for every launch
// (227 KiB, the per-block maximum), since the attribute is per function and shared
// by all host threads.
constexpr int kMaxDynSmem = 227 * 1024;

// One axis pass as a dense contraction on the tensor cores (FP32 data, BF16
// operands, tcgen05).  A: the R x Kp transform matrix (zero-padded; Kp = L rounded up to
// 32, on x after the shift below; R = Kp, on x Kp rounded up to 128) in 32-column
// chunks, each in the shared-memory core-matrix order (element (m, jj) of chunk c at
// c R 32 + (m>>3) 256 + (jj>>3) 64 + (m&7) 8 + (jj&7), in BF16 elements); on the x axis
// rows and columns are shifted by lo mod 4 (the pass indexes nodes from lo rounded down
// to a multiple of 4).  A2: the inverse z matrix of the fused z pass, same layout.
struct TcPassParams {
  const float* in[3];
  float* out[3];
  const float* base[3];
  const float* base_lo[3];
  float* out_lo[3];
  int axis;
  int N[3];
  long long stride[3];
  int lo[3], L[3], Kp[3];
  const uint16_t* A[3];
  const uint16_t* A2[3];
  float scale[3];
  int fused;
  const float* S2[3][3];
  const float* C2[3][3];
  int flo[3][3], fL[3][3];
  float hf[3];
  float two_mu0, lam0;
  int tetra;
  float gscale[3];
  int* err;  // set to 1 by a CTA whose wait on the tensor cores timed out
  const int* stop;  // device flag: nonzero once the load step has stopped (the launch does nothing)
};
cudaError_t launch_pass_tc(const TcPassParams& P, cudaStream_t s);
// Whether a transform of padded length Kp along `axis` fits one tensor-core CTA.
bool pass_tc_fits(int Kp, int axis);
// Rows of one matrix in the tensor-core chunk layout (x: Kp padded to a multiple of 128).
int pass_tc_rows(int Kp, int axis);

// One axis pass as a dense contraction on the tensor cores with TF32 operands (tcgen05
// kind::tf32, FP32 data read as is, FP32 accumulation in TMEM).  A: the R x Kp transform
// matrix (zero-padded; Kp = L rounded up to 32, on x after the shift by lo mod 4; R = Kp,
// on x Kp rounded up to 128) in 32-column chunks, each in the K-major core-matrix order of
// FP32 elements: element (m, jj) of chunk c at c R 32 + (m>>3) 256 + (jj>>2) 32 + (m&7) 4
// + (jj&3).  mode 0: out = scale T in; mode 1 (x axis): out = base + scale T in, as an
// unevaluated hi + lo pair when out_lo is set; mode 2 (z axis): the forward result times the
// B0 / 2 mu0 Green factor -gscale / den (0 where den is null).  On y and z a transform of
// 257 outputs (DCT-I over 256 intervals) runs the first Kn = 256 on the tensor cores (R = 256
// rows, two accumulators fit TMEM) and the last as a dot product of the FP32 tile with the
// matrix row xrow (K positions, FP32) in the producers.
struct TfPassParams {
  // TMA descriptors of the input components (filled by launch_pass_tf32): x axis a 2D tensor
  // {row pitch, N2 * N3 rows} in 32 x 128 boxes with the 128-byte swizzle; y and z axes a 3D
  // tensor {row pitch, N2, N3} in boxes of 128 x values by 32 rows along the axis
  CUtensorMap tmap[3];
  const float* in[3];
  float* out[3];
  const float* base[3];
  const float* base_lo[3];
  float* out_lo[3];
  int axis, mode;
  int N[3];
  long long stride[3];
  int lo[3], L[3], Kp[3];
  int Kn[3];             // outputs contracted on the tensor cores (Kp, or 256 with xrow)
  const float* xrow[3];  // y, z: the matrix row of output 256 when L = 257 (else null)
  const float* A[3];
  float scale[3];
  const float* S2[3][3];
  const float* C2[3][3];
  int flo[3][3], fL[3][3];
  float hf[3];
  float two_mu0, lam0;
  int tetra;
  float gscale[3];
  int* err;  // set to 1 by a CTA whose bounded wait on the tensor-core pipeline gave up
  const int* stop;  // device flag: nonzero once the load step has stopped (the launch does nothing)
};
cudaError_t launch_pass_tf32(const TfPassParams& P, cudaStream_t s);
bool pass_tf32_fits(int Kp, int axis, int xtra = 0);
int pass_tf32_rows(int Kp, int axis);

// Green factor on a spectral field (standalone step).
template <typename T>
struct GreenParams {
  T* f[3];
  int N[3];
  long long sy, sz;
  const T* S2[3][3];
  const T* C2[3][3];
  int flo[3][3], fL[3][3];
  T hf[3];
  T two_mu0, lam0;
  int tetra;
  T gscale[3];
};

// The C0 Green operator at every node position (fftm_c0.cu): the three components' DCT-I /
// DST-I coefficients of one position couple through v (v_q = tau_q (xi_H)_q).
template <typename T>
struct C0Params {
  T* f[3];                  // in place: p_hat in, u_hat out
  int N[3];
  long long sy, sz;
  int lo[3][3], hi[3][3];   // node-position range [lo, hi) of component q along axis a
  const T* s[3];            // sin(xi_a / 2) at node positions 0 .. N_a - 1 (xi = pi m / n_a)
  const T* c[3];            // cos(xi_a / 2), exact zero at m = n_a
  T hf[3];                  // 2 / h_a
  T tau[3];                 // -1: u_q symmetric about the faces normal to q (DCT-I), +1: anti-symmetric
  T two_mu0, beta;          // beta = lambda0 / (2 mu0 + lambda0)
  T lam0;
  int tetra;                // TETRA2: the second coupling vector w (w_q = tau_q xi'_q)
  T gscale[3];              // normalisation of the transforms (and the sign of the update)
  const int* stop;
};

// ---- launchers (return cudaError_t of the launch) ----
template <typename T>
cudaError_t launch_pass(const PassParams<T>& P, int maxM, int maxL, int maxn, cudaStream_t s);
template <typename T>
cudaError_t launch_green_c0(const C0Params<T>& P, cudaStream_t s);
template <typename T>
cudaError_t launch_residual(const ResParams<T>& P, int tetra, bool with_p, cudaStream_t s, int* blocks_out);
template <typename T>
int residual_blocks(const ResParams<T>& P, int tetra);
// Whether the residual of these parameters has the one-pass form (small-strain elastic laws,
// plain form) besides the two-pass one.
template <typename T>
bool residual_one_pass(const ResParams<T>& P);
template <typename T>
cudaError_t launch_green(const GreenParams<T>& P, cudaStream_t s);
// a9: recompute the return (J2, crystal plasticity) at every voxel point from the
// current u^f and the state of the step, and store the returned state in `out`.
template <typename T>
cudaError_t launch_commit(const ResParams<T>& P, int tetra, T* out, cudaStream_t s);
// The committed state as (eps^p, p) = (sym G_n - e_n, p_n) (out != null), or the
// elastic strain e_n = sym G_n - eps^p from a given (eps^p, p) (in != null); G_n is
// the total gradient at the commit, from P.u = u^f_n and P.Gs, P.Qc = the load at
// the commit.  Dense layout [r][7][voxel]; zero outside J2 voxels.
template <typename T>
cudaError_t launch_state_io(const ResParams<T>& P, int tetra, T* out, const T* in, cudaStream_t s);

cudaError_t launch_reduce_norms(const double* partial, int nblocks, int nvals, double* out, cudaStream_t s,
                                const int* stop = nullptr);
// Control block of a load step whose convergence is decided on the device (Algorithm 1's
// test, Eq. equilibrium_condition): ctl[0] stop (0 running, 1 converged, 2 diverged,
// 3 iteration limit), ctl[1] the iteration to check next, ctl[2] the iteration checked last.
// k_check reads S_D, S_P from sums, records err at err_hist[m] and stops the step or moves on.
cudaError_t launch_check(const double* sums, int* ctl, double* err_hist, double tol, int max_iter, double h1,
                         cudaStream_t s);

template <typename T>
cudaError_t launch_axpy_fields(T* const dst[3], const T* const a[3], const T* const b[3], T alpha,
                               long long count, cudaStream_t s);  // dst = a + alpha b
template <typename T>
cudaError_t launch_copy_fields(T* const dst[3], const T* const src[3], long long count, cudaStream_t s);
// Anderson on (u^k, D^k), newest couple last: normal matrix of D_k - D_last and
// right-hand side <D_k - D_last, D_last>, per block (9 doubles).
template <typename T>
cudaError_t launch_gram(const T* const D[4][3], int m, long long count, double* partial, int nblocks,
                        cudaStream_t s, const int* stop = nullptr);
// accepted: the step's flag array, indexed by ctl[2] when ctl is given (device-decided loop),
// else accepted[0].
cudaError_t launch_anderson_solve(const double* partial, int nblocks, int m, double pivot_tol, double* coef,
                                  int* accepted, cudaStream_t s, const int* ctl = nullptr);
// Dbar = sum c_k D_k -> dst;  ubar = u_last + sum_k c_k (u_k - u_last) -> (bh, bl)
template <typename T>
cudaError_t launch_combine(T* const dst[3], T* const bh[3], T* const bl[3], const T* const D[4][3],
                           const T* const uh[4][3], const T* const ul[4][3], int m, const double* coef,
                           long long count, cudaStream_t s, const int* stop = nullptr);
template <typename T>
cudaError_t launch_voxel_fields(const ResParams<T>& P, int tetra, T* grad_out, T* stress_out, cudaStream_t s);
template <typename T>
cudaError_t launch_pack(const T* const src[3], T* dst, int N1, int N2, int N3, long long sy, long long sz,
                        int unpack, cudaStream_t s);
template <typename T>
cudaError_t launch_mask(T* const f[3], const int lo[3][3], const int hi[3][3], int N1, int N2, int N3,
                        long long sy, long long sz, cudaStream_t s);

int gram_blocks(long long count);
// Measured FMA throughput of the current device (FLOP/s, an FMA counting two), FP64 or FP32.
double fma_peak_flops(int fp64);

// Asynchronous global -> shared copies (cp.async, Ampere and later): the copy
// is issued without a register round trip, so a thread can keep many loads in
// flight; cp_async_wait_all() + __syncthreads() make them visible.
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  if (sizeof(T) == 8) cp_async_8(smem, gmem);
  else cp_async_4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// wait until at most one committed group is still in flight
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
template <typename T>
cudaError_t launch_stats(const ResParams<T>& P, int tetra, double* partial, int nblocks, cudaStream_t s);

}  // namespace fftm
