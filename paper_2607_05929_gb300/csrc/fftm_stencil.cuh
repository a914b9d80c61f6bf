// Fixed-point residual: gradient -> constitutive law -> divergence
// (Algorithm 1: grad u, P, D = div P + D*, the error; Eq. div_pol for p).
//
// Two passes over the grid.  k_stress (one thread per voxel) evaluates the
// gradient at the voxel point(s) (HEX1: Eqs. D1HG-D3HG; TETRA2: Eqs.
// D1T1T2G-D3T1T2G) and the law, and stores P (for the test variant also
// tau = R0 : grad u^f - P with B0 = 2 mu0 G + lambda0 G (.) I, Sec. 2.6.3, or C0 = 2 mu0 G + lambda0 tr(G) I, Sec. 2.6.1).
// k_div (one thread per node) applies Remark 1 -- node m reads the voxels
// m + o - 1 with the same signs -- to get D = div P (and p = div tau), written
// for the transformed node components (dismissed ones get 0).  FP64 block
// partials of S_D = sum D^2 and S_P = sum ||P||^2 / n_ppv go to `partial`.
//
// Stencil sums are formed as sums of differences of neighbouring values
// (u(o + e_i) - u(o) for HEX1; the paper's pairs for TETRA2), which are exact
// or nearly so in floating point for smooth fields, so the gradient carries
// the relative precision of the arithmetic instead of that of |u|.  In FP32
// the displacement is held as an unevaluated sum hi + lo of two floats (its
// low part carries what FP32 drops); both parts are differenced.  The norm
// partials are summed in the field precision over short runs and in FP64
// across runs (FP64 throughput is a small fraction of FP32 on this GPU).
//
// TETRA2: tetrahedron T1 uses the four even-parity corners of the voxel, T2 the
// four odd-parity ones; along axis i the paper's two differences pair each
// corner c with o_i = 0 with c ^ (e_i + e_{i+1 mod 3}), over 2 h_i.  HEX1 pairs
// c with c + e_i over 4 h_i.  The residual D = 1/2 (div_T2 P^T1 + div_T1 P^T2)
// reads from the voxel at node offset o the T1 point for odd-parity o and the
// T2 point for even o, with weight sign / (4 h_i) -- the HEX1 weights.
//
// Ghost voxels (outside non-periodic faces) are never stored: a read is
// redirected to the mirror voxel inside, with the sign sigma(u_q, face) *
// (-1 if i is the face normal) on component (i, q), and with T1 <-> T2
// swapped once per face crossed (Sec. 2.2, Sec. 2.5.2).  Periodic axes wrap.
#pragma once
// Included by fftm_stencil_f32.cu and fftm_stencil_f64.cu, which instantiate the launchers for
// one precision each (two translation units that compile in parallel).
#include <algorithm>

#include "fftm_internal.cuh"

namespace fftm {

enum { LAW_ISO = 0, LAW_CUBIC = 1, LAW_J2 = 2, LAW_B0 = 3, LAW_SVK = 4, LAW_NEOHOOKE = 5, LAW_CP = 6, LAW_LOGJ2 = 7 };

// Symmetric tensor (11, 22, 33, 23, 13, 12) -> C : E with the Mandel 6x6 stiffness stored as
// its upper triangle row-major in c[0..20].
template <typename T>
__device__ __forceinline__ void mandel_apply(const T* __restrict__ c, const T e[6], T s[6]) {
  const T r2 = T(1.41421356237309504880), ir2 = T(0.70710678118654752440);
  const T em[6] = {e[0], e[1], e[2], r2 * e[3], r2 * e[4], r2 * e[5]};
  T sm[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  int k = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = a; b < 6; ++b) {
      const T v = __ldg(c + k++);
      sm[a] += v * em[b];
      if (b != a) sm[b] += v * em[a];
    }
  s[0] = sm[0];
  s[1] = sm[1];
  s[2] = sm[2];
  s[3] = ir2 * sm[3];
  s[4] = ir2 * sm[4];
  s[5] = ir2 * sm[5];
}

// A law constant: read through the read-only cache on the device, plainly on the host (the
// host instantiation serves fftm_host_log_j2).
template <typename T>
__host__ __device__ __forceinline__ T ldc(const T* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// Finite strain (Sec. 3.1.2, Appendix B): F = 1 + H with H_qi = G[i*3+q]; the
// Green-Lagrange strain E = (H + H^T + H^T H) / 2 is formed from H so that it keeps
// its relative precision.  S[i*3+q] = P_qi with P = F Pi.
template <typename T>
__host__ __device__ __forceinline__ void green_lagrange(const T G[9], T H[3][3], T E[6]) {
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i) H[q][i] = G[i * 3 + q];
  auto e = [&](int i, int j) {
    return T(0.5) * (H[i][j] + H[j][i] + H[0][i] * H[0][j] + H[1][i] * H[1][j] + H[2][i] * H[2][j]);
  };
  E[0] = e(0, 0);
  E[1] = e(1, 1);
  E[2] = e(2, 2);
  E[3] = e(1, 2);
  E[4] = e(0, 2);
  E[5] = e(0, 1);
}

template <typename T>
__host__ __device__ __forceinline__ void first_piola(const T H[3][3], const T Pi[6], T S[9]) {
  const T M[3][3] = {{Pi[0], Pi[5], Pi[4]}, {Pi[5], Pi[1], Pi[3]}, {Pi[4], Pi[3], Pi[2]}};
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i) S[i * 3 + q] = M[q][i] + H[q][0] * M[0][i] + H[q][1] * M[1][i] + H[q][2] * M[2][i];
}

// Neo-Hookean (Appendix B): Pi = mu J^(-2/3) dev(C) C^-1 + K (J - 1) J C^-1 with C = 1 + 2E,
// J - 1 = tr H + ((tr H)^2 - tr(H^2)) / 2 + det H; c = (mu, K).
template <typename T>
__device__ __forceinline__ void neo_hooke(const T* __restrict__ c, const T G[9], T S[9]) {
  const T mu = __ldg(c), K = __ldg(c + 1);
  T H[3][3], E[6];
  green_lagrange<T>(G, H, E);
  const T trH = H[0][0] + H[1][1] + H[2][2];
  T trH2 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trH2 += H[i][j] * H[j][i];
  const T detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) - H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                 H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
  const T Jm1 = trH + T(0.5) * (trH * trH - trH2) + detH;
  const T J = T(1) + Jm1;
  // C = 1 + 2E and its inverse (adjugate / det C, det C = J^2)
  const T C00 = T(1) + T(2) * E[0], C11 = T(1) + T(2) * E[1], C22 = T(1) + T(2) * E[2];
  const T C12 = T(2) * E[3], C02 = T(2) * E[4], C01 = T(2) * E[5];
  const T ij2 = T(1) / (J * J);
  const T I00 = (C11 * C22 - C12 * C12) * ij2, I11 = (C00 * C22 - C02 * C02) * ij2, I22 = (C00 * C11 - C01 * C01) * ij2;
  const T I12 = (C02 * C01 - C00 * C12) * ij2, I02 = (C01 * C12 - C02 * C11) * ij2, I01 = (C02 * C12 - C01 * C22) * ij2;
  const T Ci[3][3] = {{I00, I01, I02}, {I01, I11, I12}, {I02, I12, I22}};
  const T tE = (E[0] + E[1] + E[2]) * T(2.0 / 3.0);
  const T Dv[3][3] = {{T(2) * E[0] - tE, T(2) * E[5], T(2) * E[4]},
                      {T(2) * E[5], T(2) * E[1] - tE, T(2) * E[3]},
                      {T(2) * E[4], T(2) * E[3], T(2) * E[2] - tE}};
  const T a = mu * exp(T(-2.0 / 3.0) * log1p(Jm1)), b = K * Jm1 * J;
  auto pi = [&](int i, int j) {
    return a * (Dv[i][0] * Ci[0][j] + Dv[i][1] * Ci[1][j] + Dv[i][2] * Ci[2][j]) + b * Ci[i][j];
  };
  const T Pi[6] = {pi(0, 0), pi(1, 1), pi(2, 2), pi(1, 2), pi(0, 2), pi(0, 1)};
  first_piola<T>(H, Pi, S);
}


// ---- FCC crystal plasticity, finite strain (Sec. 3.4) ----------------------------
// The 12 {111}<110> systems in the crystal frame (unnormalised plane normal, slip
// direction); the normalisation 1/sqrt(6) of m (x) n is applied at use.
static __constant__ signed char c_fcc_sys[12][6] = {
    {1, 1, 1, 0, 1, -1},  {1, 1, 1, 1, 0, -1},  {1, 1, 1, 1, -1, 0},  {-1, 1, 1, 0, 1, -1},
    {-1, 1, 1, 1, 0, 1},  {-1, 1, 1, 1, 1, 0},  {1, -1, 1, 0, 1, 1},  {1, -1, 1, 1, 0, -1},
    {1, -1, 1, 1, 1, 0},  {1, 1, -1, 0, 1, 1},  {1, 1, -1, 1, 0, 1},  {1, 1, -1, 1, -1, 0}};

// (1 + K)^-1 - 1 for a small K, without forming 1 + K: with Cayley-Hamilton,
// adj(1 + K) = 1 + D, D = (tr K + c2) 1 - (1 + tr K) K + K^2, det(1 + K) = 1 + d,
// d = tr K + c2 + det K, c2 = ((tr K)^2 - tr K^2) / 2; the result is (D - d 1) / (1 + d).
template <typename T>
__device__ __forceinline__ void inv_minus_identity(const T K[9], T Y[9]) {
  const T tr = K[0] + K[4] + K[8];
  T K2[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) K2[i * 3 + j] = K[i * 3] * K[j] + K[i * 3 + 1] * K[3 + j] + K[i * 3 + 2] * K[6 + j];
  const T trK2 = K2[0] + K2[4] + K2[8];
  const T c2 = T(0.5) * (tr * tr - trK2);
  const T det = K[0] * (K[4] * K[8] - K[5] * K[7]) - K[1] * (K[3] * K[8] - K[5] * K[6]) + K[2] * (K[3] * K[7] - K[4] * K[6]);
  const T d = tr + c2 + det;
  const T inv = T(1) / (T(1) + d);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T Dm = ((i % 4 == 0) ? (tr + c2) : T(0)) - (T(1) + tr) * K[i] + K2[i];
    Y[i] = (Dm - ((i % 4 == 0) ? d : T(0))) * inv;
  }
}

// (1 + X)(1 + Y) - 1 = X + Y + X Y
template <typename T>
__device__ __forceinline__ void compose_minus_identity(const T X[9], const T Y[9], T W[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      W[i * 3 + j] = X[i * 3 + j] + Y[i * 3 + j] + X[i * 3] * Y[j] + X[i * 3 + 1] * Y[3 + j] + X[i * 3 + 2] * Y[6 + j];
}

// One implicit increment at a voxel point (Kalidindi, Bronkhorst and Anand 1992):
// unknown second Piola-Kirchhoff Pi (6 components 11, 22, 33, 23, 13, 12),
//   R(Pi) = Pi - Pi_tr + sum_s dgamma_s(tau_s) C : sym(A P_s),  tau_s = Pi : P_s,
//   dgamma_s = dt gdot0 |tau_s / tau_c|^n sign(tau_s),  tau_c = Voce(Gamma_n),
// Newton from the trial stress scaled onto the yield surface of the most stressed
// system, with backtracking on max |R|; then F^p = (1 + sum dgamma_s P_s) F^p_n,
// Gamma += sum |dgamma_s|, P = F^e Pi F^p^-T.  State st = (F^p - 1 row-major, Gamma).
// c = Mandel C (21), gdot0, n, tau0, tau_inf, h0, dt, R (crystal -> sample, row-major).
template <typename T>
__device__ void cp_eval(const T* __restrict__ c, const T G[9], const T st[10], T S[9], T* stn) {
  const T gdot0 = __ldg(c + 21), nexp = __ldg(c + 22), tau0 = __ldg(c + 23), tinf = __ldg(c + 24);
  const T h0 = __ldg(c + 25), dt = __ldg(c + 26);
  T Rm[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Rm[i] = __ldg(c + 27 + i);
  // Schmid tensors, symmetric parts (6 components) and full (9)
  T sP[12][6], Pf[12][9];
  const T inv6 = T(0.40824829046386301637);  // 1 / sqrt(6)
#pragma unroll
  for (int s = 0; s < 12; ++s) {
    T nv[3], mv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      nv[i] = Rm[i * 3] * T(c_fcc_sys[s][0]) + Rm[i * 3 + 1] * T(c_fcc_sys[s][1]) + Rm[i * 3 + 2] * T(c_fcc_sys[s][2]);
      mv[i] = Rm[i * 3] * T(c_fcc_sys[s][3]) + Rm[i * 3 + 1] * T(c_fcc_sys[s][4]) + Rm[i * 3 + 2] * T(c_fcc_sys[s][5]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Pf[s][i * 3 + j] = inv6 * mv[i] * nv[j];
    sP[s][0] = Pf[s][0];
    sP[s][1] = Pf[s][4];
    sP[s][2] = Pf[s][8];
    sP[s][3] = T(0.5) * (Pf[s][5] + Pf[s][7]);
    sP[s][4] = T(0.5) * (Pf[s][2] + Pf[s][6]);
    sP[s][5] = T(0.5) * (Pf[s][1] + Pf[s][3]);
  }
  // trial elastic state: W = F F^p_n^-1 - 1, E_tr = (W + W^T + W^T W) / 2, A = 1 + 2 E_tr
  T H[9], Y[9], W[9];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i) H[q * 3 + i] = G[i * 3 + q];
  inv_minus_identity<T>(st, Y);
  compose_minus_identity<T>(H, Y, W);
  auto ew = [&](int i, int j) {
    return T(0.5) * (W[i * 3 + j] + W[j * 3 + i] + W[i] * W[j] + W[3 + i] * W[3 + j] + W[6 + i] * W[6 + j]);
  };
  const T Etr[6] = {ew(0, 0), ew(1, 1), ew(2, 2), ew(1, 2), ew(0, 2), ew(0, 1)};
  T Ptr[6];
  mandel_apply<T>(c, Etr, Ptr);
  // C : sym(A P_s) = C : sym(P_s) + 2 C : sym(E_tr P_s)
  T Cs[12][6];
  {
    const T Em[3][3] = {{Etr[0], Etr[5], Etr[4]}, {Etr[5], Etr[1], Etr[3]}, {Etr[4], Etr[3], Etr[2]}};
#pragma unroll
    for (int s = 0; s < 12; ++s) {
      T B[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          B[i][j] = Em[i][0] * Pf[s][j] + Em[i][1] * Pf[s][3 + j] + Em[i][2] * Pf[s][6 + j];
      const T v[6] = {sP[s][0] + T(2) * B[0][0], sP[s][1] + T(2) * B[1][1], sP[s][2] + T(2) * B[2][2],
                      sP[s][3] + (B[1][2] + B[2][1]), sP[s][4] + (B[0][2] + B[2][0]), sP[s][5] + (B[0][1] + B[1][0])};
      mandel_apply<T>(c, v, Cs[s]);
    }
  }
  const T gam_n = st[9];
  const T tauc = tinf > tau0 ? tau0 + (tinf - tau0) * (T(1) - exp(-h0 * gam_n / (tinf - tau0))) : tau0;
  auto tau_of = [&](const T Pi[6], int s) {
    return Pi[0] * sP[s][0] + Pi[1] * sP[s][1] + Pi[2] * sP[s][2] +
           T(2) * (Pi[3] * sP[s][3] + Pi[4] * sP[s][4] + Pi[5] * sP[s][5]);
  };
  auto slip = [&](T tau, T* ddg) {
    const T x = tau / tauc, ax = fabs(x);
    const T pw = ax > T(0) ? exp((nexp - T(1)) * log(ax)) : T(0);  // |x|^(n-1)
    if (ddg) *ddg = dt * gdot0 * nexp * pw / tauc;
    return copysign(dt * gdot0 * pw * ax, x);
  };
  auto resid = [&](const T Pi[6], T R[6]) {
    T m = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) R[k] = Pi[k] - Ptr[k];
    for (int s = 0; s < 12; ++s) {
      const T dg = slip(tau_of(Pi, s), nullptr);
#pragma unroll
      for (int k = 0; k < 6; ++k) R[k] += dg * Cs[s][k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) m = fmax(m, fabs(R[k]));
    return m;
  };
  T taumax = T(0), scale = tauc;
  for (int s = 0; s < 12; ++s) taumax = fmax(taumax, fabs(tau_of(Ptr, s)));
#pragma unroll
  for (int k = 0; k < 6; ++k) scale = fmax(scale, fabs(Ptr[k]));
  const T s0 = taumax > tauc ? tauc / taumax : T(1);
  T Pi[6], R[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) Pi[k] = s0 * Ptr[k];
  T rn = resid(Pi, R);
  // FP32: about two units in the last place of the largest stress component, the level at
  // which the residual itself is rounding; FP64: the oracle's tolerance
  const T tol = (sizeof(T) == 8 ? T(1e-12) : T(1.2e-7)) * scale;
  for (int it = 0; it < 200 && rn > tol; ++it) {
    // Jacobian: 1 + sum_s ddgamma_s C_s (x) dtau_s/dPi
    T J[6][7];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
#pragma unroll
      for (int b = 0; b < 6; ++b) J[a][b] = (a == b) ? T(1) : T(0);
      J[a][6] = -R[a];
    }
    for (int s = 0; s < 12; ++s) {
      T ddg;
      slip(tau_of(Pi, s), &ddg);
      const T g[6] = {sP[s][0], sP[s][1], sP[s][2], T(2) * sP[s][3], T(2) * sP[s][4], T(2) * sP[s][5]};
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = 0; b < 6; ++b) J[a][b] += ddg * Cs[s][a] * g[b];
    }
    // Gaussian elimination with partial pivoting
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      int piv = k;
      for (int a = k + 1; a < 6; ++a)
        if (fabs(J[a][k]) > fabs(J[piv][k])) piv = a;
      if (piv != k)
        for (int b = 0; b < 7; ++b) {
          const T t = J[k][b];
          J[k][b] = J[piv][b];
          J[piv][b] = t;
        }
      const T ip = T(1) / J[k][k];
      for (int a = k + 1; a < 6; ++a) {
        const T f = J[a][k] * ip;
        for (int b = k; b < 7; ++b) J[a][b] -= f * J[k][b];
      }
    }
    T d[6];
    for (int k = 5; k >= 0; --k) {
      T v = J[k][6];
      for (int b = k + 1; b < 6; ++b) v -= J[k][b] * d[b];
      d[k] = v / J[k][k];
    }
    // backtracking on max |R|
    T step = T(1), Pn[6], Rn[6], rnew = rn;
    for (int bt = 0; bt < (sizeof(T) == 8 ? 60 : 24); ++bt) {
#pragma unroll
      for (int k = 0; k < 6; ++k) Pn[k] = Pi[k] + step * d[k];
      rnew = resid(Pn, Rn);
      if (rnew < rn || step <= T(1e-12)) break;
      step *= T(0.5);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      Pi[k] = Pn[k];
      R[k] = Rn[k];
    }
    if (!(rnew < rn)) break;  // no descent left at this precision
    rn = rnew;
  }
  // plastic update: K' = (1 + L)(1 + K) - 1, L = sum dgamma_s P_s; Gamma += sum |dgamma_s|
  T L[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)}, dgam = T(0);
  for (int s = 0; s < 12; ++s) {
    const T dg = slip(tau_of(Pi, s), nullptr);
    dgam += fabs(dg);
#pragma unroll
    for (int i = 0; i < 9; ++i) L[i] += dg * Pf[s][i];
  }
  T K1[9], Y1[9], W1[9];
  compose_minus_identity<T>(L, st, K1);
  inv_minus_identity<T>(K1, Y1);
  compose_minus_identity<T>(H, Y1, W1);
  // P = (1 + W1) Pi (1 + Y1)^T; S[i*3+q] = P_qi
  const T M[3][3] = {{Pi[0], Pi[5], Pi[4]}, {Pi[5], Pi[1], Pi[3]}, {Pi[4], Pi[3], Pi[2]}};
  T FM[3][3];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      FM[q][j] = M[q][j] + W1[q * 3] * M[0][j] + W1[q * 3 + 1] * M[1][j] + W1[q * 3 + 2] * M[2][j];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      S[i * 3 + q] = FM[q][i] + FM[q][0] * Y1[i * 3] + FM[q][1] * Y1[i * 3 + 1] + FM[q][2] * Y1[i * 3 + 2];
  if (stn) {
#pragma unroll
    for (int i = 0; i < 9; ++i) stn[i] = K1[i];
    stn[9] = gam_n + dgam;
  }
}

// Eigen-decomposition of a symmetric 3x3 tensor A (11, 22, 33, 23, 13, 12) by cyclic
// Jacobi rotations (each rotation zeroes one off-diagonal entry; the tangent of the angle is
// taken as the smaller root of t^2 + 2 th t - 1 = 0, th = (a_qq - a_pp) / (2 a_pq), and the
// other entries are updated through tau = s / (1 + c) to limit cancellation).  Returns the
// eigenvalues w and the eigenvectors as the columns of V (row-major).  The sweep count is
// fixed: convergence is quadratic, so 5 (FP32) or 6 (FP64) sweeps leave the off-diagonal at
// rounding level for any input; an entry that is already zero is skipped.
template <typename T>
__host__ __device__ void sym_eig3(const T A6[6], T w[3], T V[9]) {
  T a[3][3] = {{A6[0], A6[5], A6[4]}, {A6[5], A6[1], A6[3]}, {A6[4], A6[3], A6[2]}};
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? T(1) : T(0);
  constexpr int SWEEPS = sizeof(T) == 8 ? 6 : 5;
  for (int sw = 0; sw < SWEEPS; ++sw) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int p = k == 2 ? 1 : 0, q = k == 0 ? 1 : 2, r = 3 - p - q;
      const T apq = a[p][q];
      if (apq == T(0)) continue;
      const T th = (a[q][q] - a[p][p]) / (T(2) * apq);
      const T t = copysign(T(1), th) / (fabs(th) + sqrt(th * th + T(1)));  // th^2 = inf gives t = 0
      const T c = T(1) / sqrt(t * t + T(1)), sn = t * c, tau = sn / (T(1) + c);
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = T(0);
      const T g = a[r][p], h = a[r][q];
      a[r][p] = a[p][r] = g - sn * (h + g * tau);
      a[r][q] = a[q][r] = h + sn * (g - h * tau);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T vg = V[i * 3 + p], vh = V[i * 3 + q];
        V[i * 3 + p] = vg - sn * (vh + vg * tau);
        V[i * 3 + q] = vh + sn * (vg - vh * tau);
      }
    }
  }
  w[0] = a[0][0];
  w[1] = a[1][1];
  w[2] = a[2][2];
}

// Perfect von Mises plasticity in the logarithmic strain space (Sec. 3.2, the porous
// medium; reading: T is the stress conjugate to the Hencky strain, Miehe, Apel and
// Lambrecht 2002).  H = log C / 2 with C = F^T F = 1 + 2E; H = H^e + H^p; trial
// H^e = H - H^p_n, T = 2 mu dev H^e + K tr H^e 1; on f = sqrt(3/2) |dev T| - sigma0 > 0 the
// backward-Euler return scales dev T onto the yield surface, dp = f / (3 mu), H^p += dp
// 3/2 dev T_tr / |.|_eq.  S = T : d log C / d C: in the eigenbasis of C, S_ab = theta_ab T_ab
// with theta_ab = (log w_a - log w_b) / (w_a - w_b) (1 / w_a on the diagonal); P = F S.
// The eigenvalues are taken from E (w_a = 1 + 2 e_a), so log w_a = log1p(2 e_a) and the
// divided differences, r = 2 (e_a - e_b) / w_b, keep their relative precision.
// c = (lambda, mu, sigma0); st = (H^p 11, 22, 33, 23, 13, 12; p); stn: the returned state.
template <typename T>
__host__ __device__ void log_j2_eval(const T* __restrict__ c, const T G[9], const T st[7], T S[9], T* stn) {
  const T lam = ldc(c), mu = ldc(c + 1), sig0 = ldc(c + 2);
  const T K = lam + T(2.0 / 3.0) * mu;
  T H[3][3], E[6];
  green_lagrange<T>(G, H, E);
  T e[3], V[9];
  sym_eig3<T>(E, e, V);
  T hl[3], w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w[a] = T(1) + T(2) * e[a];
    hl[a] = T(0.5) * log1p(T(2) * e[a]);
  }
  constexpr int I6[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  T He[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int i = I6[k][0], j = I6[k][1];
    He[k] = (V[i * 3] * hl[0] * V[j * 3] + V[i * 3 + 1] * hl[1] * V[j * 3 + 1] + V[i * 3 + 2] * hl[2] * V[j * 3 + 2]) -
            st[k];
  }
  const T tr = He[0] + He[1] + He[2], m = tr * T(1.0 / 3.0), m2 = T(2) * mu;
  const T s6[6] = {m2 * (He[0] - m), m2 * (He[1] - m), m2 * (He[2] - m), m2 * He[3], m2 * He[4], m2 * He[5]};
  const T ss = s6[0] * s6[0] + s6[1] * s6[1] + s6[2] * s6[2] + T(2) * (s6[3] * s6[3] + s6[4] * s6[4] + s6[5] * s6[5]);
  const T seq = sqrt(T(1.5) * ss);
  const T f = seq - sig0;
  T scale = T(1), dp = T(0);
  if (f > T(0)) {
    dp = f / (T(3) * mu);
    scale = sig0 / seq;
  }
  if (stn) {
    const T g = f > T(0) ? dp * T(1.5) / seq : T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) stn[k] = st[k] + g * s6[k];
    stn[6] = st[6] + dp;
  }
  const T kt = K * tr;
  const T Tm[3][3] = {{scale * s6[0] + kt, scale * s6[5], scale * s6[4]},
                      {scale * s6[5], scale * s6[1] + kt, scale * s6[3]},
                      {scale * s6[4], scale * s6[3], scale * s6[2] + kt}};
  // St = theta o (V^T T V), then S = V St V^T
  T TV[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int b = 0; b < 3; ++b) TV[i][b] = Tm[i][0] * V[b] + Tm[i][1] * V[3 + b] + Tm[i][2] * V[6 + b];
  T St[3][3];
  const T near = sizeof(T) == 8 ? T(1e-10) : T(1e-30);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T tt = V[a] * TV[0][b] + V[3 + a] * TV[1][b] + V[6 + a] * TV[2][b];
      const T r = T(2) * (e[a] - e[b]) / w[b];
      const T th = fabs(r) < near ? T(2) / (w[a] + w[b]) : log1p(r) / (w[b] * r);
      St[a][b] = th * tt;
    }
  T Pi[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int i = I6[k][0], j = I6[k][1];
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) acc += V[i * 3 + a] * St[a][b] * V[j * 3 + b];
    Pi[k] = acc;
  }
  first_piola<T>(H, Pi, S);
}

// Small-strain law on the total gradient G[i*3+q]; P returned as 9 components.
template <typename T>
__device__ __forceinline__ void law_eval(int law, const T* __restrict__ c, const T G[9], T Pout[9]) {
  const T e00 = G[0], e11 = G[4], e22 = G[8];
  const T e12 = T(0.5) * (G[5] + G[7]);
  const T e02 = T(0.5) * (G[2] + G[6]);
  const T e01 = T(0.5) * (G[1] + G[3]);
  if (law == LAW_CUBIC) {
    // Mandel 6x6 stiffness, upper triangle row-major in c[0..20]
    const T r2 = T(1.41421356237309504880);
    const T em[6] = {e00, e11, e22, r2 * e12, r2 * e02, r2 * e01};
    T sm[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    int k = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) {
        const T v = __ldg(c + k++);
        sm[a] += v * em[b];
        if (b != a) sm[b] += v * em[a];
      }
    const T ir2 = T(0.70710678118654752440);
    Pout[0] = sm[0];
    Pout[4] = sm[1];
    Pout[8] = sm[2];
    Pout[5] = Pout[7] = ir2 * sm[3];
    Pout[2] = Pout[6] = ir2 * sm[4];
    Pout[1] = Pout[3] = ir2 * sm[5];
  } else if (law == LAW_SVK) {  // St-Venant-Kirchhoff, Pi = C : E (Sec. 3.1.2)
    T H[3][3], E[6], Pi[6];
    green_lagrange<T>(G, H, E);
    mandel_apply<T>(c, E, Pi);
    first_piola<T>(H, Pi, Pout);
  } else if (law == LAW_NEOHOOKE) {
    neo_hooke<T>(c, G, Pout);
  } else if (law == LAW_B0) {
    const T lam = __ldg(c), mu2 = T(2) * __ldg(c + 1);
#pragma unroll
    for (int i = 0; i < 9; ++i) Pout[i] = mu2 * G[i];
    Pout[0] += lam * G[0];
    Pout[4] += lam * G[4];
    Pout[8] += lam * G[8];
  } else {  // isotropic elasticity
    const T lam = __ldg(c), mu2 = T(2) * __ldg(c + 1);
    const T tr = lam * (e00 + e11 + e22);
    Pout[0] = tr + mu2 * e00;
    Pout[4] = tr + mu2 * e11;
    Pout[8] = tr + mu2 * e22;
    Pout[5] = Pout[7] = mu2 * e12;
    Pout[2] = Pout[6] = mu2 * e02;
    Pout[1] = Pout[3] = mu2 * e01;
  }
}

// J2 plasticity with linear isotropic hardening (Sec. 3.2, small strain), radial
// return written as an increment from the committed state st = (e_n as 11, 22, 33,
// 23, 13, 12; p_n), e_n the elastic strain at the commit, for the gradient
// increment dG since the commit.  With K = lambda + 2 mu / 3, d the deviator of e_n
// and dd that of sym(dG):
//   trial von Mises stress q = 2 mu sqrt(3/2 (d + dd):(d + dd)), written as
//   q_n + dq with dq = (q^2 - q_n^2) / (q + q_n) (a small quantity);
//   yield function f = (q_n - sigma_y - H p_n) + dq; on yield dp = f / (3 mu + H)
//   and the deviator is scaled by k = 1 + km1, km1 = -3 mu dp / q;
//   P - P_n = K tr(dG) I + 2 mu (k dd + km1 d),  P_n = K tr(e_n) I + 2 mu d.
// In exact arithmetic this is the classical return on e = e_n + sym(dG); written
// this way every rounding is relative to the increment, not to the stress.
// c = (lambda, mu, sigma_y, H).  dP (may be null): P - P_n; Pf: P; stn (may be
// null): the returned state (e_{n+1} = volumetric part + k times the deviator).
template <typename T>
__device__ __forceinline__ void j2_inc(const T* __restrict__ c, const T dG[9], const T st[7], T* dP, T Pf[9],
                                       T* stn) {
  const T lam = __ldg(c), mu = __ldg(c + 1), sy = __ldg(c + 2), H = __ldg(c + 3);
  const T de[6] = {dG[0], dG[4], dG[8], T(0.5) * (dG[5] + dG[7]), T(0.5) * (dG[2] + dG[6]),
                   T(0.5) * (dG[1] + dG[3])};
  const T dtr = de[0] + de[1] + de[2], dm = dtr * T(1.0 / 3.0);
  const T trn = st[0] + st[1] + st[2], mn = trn * T(1.0 / 3.0);
  const T dd[6] = {de[0] - dm, de[1] - dm, de[2] - dm, de[3], de[4], de[5]};
  const T dn[6] = {st[0] - mn, st[1] - mn, st[2] - mn, st[3], st[4], st[5]};
  auto dot = [](const T* a, const T* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + T(2) * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
  };
  const T c2 = T(6) * mu * mu;  // 3/2 (2 mu)^2
  const T qn = sqrt(c2 * dot(dn, dn));
  const T dq2 = c2 * (T(2) * dot(dn, dd) + dot(dd, dd));
  const T q2 = qn * qn + dq2;
  const T q = q2 > T(0) ? sqrt(q2) : T(0);
  const T dq = (q + qn) > T(0) ? dq2 / (q + qn) : T(0);
  const T f = (qn - (sy + H * st[6])) + dq;
  T dp = T(0), km1 = T(0);
  if (f > T(0)) {
    dp = f / (T(3) * mu + H);
    km1 = -T(3) * mu * dp / q;
  }
  const T K = lam + T(2.0 / 3.0) * mu, m2 = T(2) * mu;
  T d6[6], p6[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    d6[i] = m2 * ((T(1) + km1) * dd[i] + km1 * dn[i]) + (i < 3 ? K * dtr : T(0));
    p6[i] = (m2 * dn[i] + (i < 3 ? K * trn : T(0))) + d6[i];
  }
  constexpr int map9[9] = {0, 5, 4, 5, 1, 3, 4, 3, 2};  // G[i*3+q] -> symmetric slot
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    Pf[i] = p6[map9[i]];
    if (dP) dP[i] = d6[map9[i]];
  }
  if (stn) {
#pragma unroll
    for (int i = 0; i < 6; ++i) stn[i] = (i < 3 ? mn + dm : T(0)) + (T(1) + km1) * (dn[i] + dd[i]);
    stn[6] = st[6] + dp;
  }
}

// Law at voxel point r of voxel v from the gradient G (elastic laws: the total
// gradient; J2: the increment since the commit).
template <typename T, int SL = 7>
__device__ __forceinline__ void point_law(const ResParams<T>& P, int law, const T* lc, const T G[9], int r,
                                          long long v, long long nvox, T Pout[9], T* stn) {
  if ((SL & 1) && law == LAW_J2) {
    const T* sp = P.state + (long long)(r * P.nst) * nvox + v;
    T st[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) st[c] = sp[c * nvox];
    j2_inc<T>(lc, G, st, nullptr, Pout, stn);
  } else if ((SL & 2) && law == LAW_CP) {
    const T* sp = P.state + (long long)(r * P.nst) * nvox + v;
    T st[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) st[c] = sp[c * nvox];
    cp_eval<T>(lc, G, st, Pout, stn);
  } else if ((SL & 4) && law == LAW_LOGJ2) {
    const T* sp = P.state + (long long)(r * P.nst) * nvox + v;
    T st[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) st[c] = sp[c * nvox];
    log_j2_eval<T>(lc, G, st, Pout, stn);
  } else {
    law_eval<T>(law, lc, G, Pout);
  }
}

// Quadratic part sum_k Q_qk m_k of u*, m = (x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2): its
// discrete gradient at voxel (vx, vy, vz), point r, worked out from the stencils'
// corners: D_i (x_a^2) = 2 x_a delta_ia at the voxel centre (both schemes);
// D_i (x_a x_b) = x_b delta_ia + x_a delta_ib, plus on the third axis c 0 for HEX1
// and -h_a h_b / (2 h_c) on T1, +h_a h_b / (2 h_c) on T2 (Eqs. D1HG-D3HG, D1T1T2G-D3T1T2G).
template <typename T, int TETRA>
__device__ __forceinline__ void add_quad(const T hh[3], const T Q[3][6], int r, int vx, int vy, int vz, T G[9]) {
  const T x0 = (T(vx) + T(0.5)) * hh[0], x1 = (T(vy) + T(0.5)) * hh[1], x2 = (T(vz) + T(0.5)) * hh[2];
  const T sg = TETRA ? (r == 0 ? T(-0.5) : T(0.5)) : T(0);
  const T k23 = sg * hh[1] * hh[2] / hh[0], k13 = sg * hh[0] * hh[2] / hh[1], k12 = sg * hh[0] * hh[1] / hh[2];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const T a = Q[q][0], b = Q[q][1], c = Q[q][2], d = Q[q][3], e = Q[q][4], f = Q[q][5];
    G[q] += T(2) * a * x0 + e * x2 + f * x1 + d * k23;
    G[3 + q] += T(2) * b * x1 + d * x2 + f * x0 + e * k13;
    G[6 + q] += T(2) * c * x2 + d * x1 + e * x0 + f * k12;
  }
}

// Gradient at point r from the 8 corner values (corner o = ox + 2 oy + 4 oz),
// as a sum of differences; ul (low parts) may be null.
template <typename T, int TETRA, bool LO>
__device__ __forceinline__ void point_grad(const T uh[3][8], const T ul[3][8], int r, const T* wg, T G[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int mask = TETRA ? ((1 << i) | (1 << ((i + 1) % 3))) : (1 << i);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T s = T(0), sl = T(0);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        if ((o >> i) & 1) continue;  // base corners have o_i = 0
        const int par = ((o & 1) + ((o >> 1) & 1) + ((o >> 2) & 1)) & 1;
        if (TETRA && ((r == 0) != (par == 0))) continue;  // T1: even corners, T2: odd corners
        s += uh[q][o ^ mask] - uh[q][o];
        if (LO) sl += ul[q][o ^ mask] - ul[q][o];
      }
      G[i * 3 + q] = wg[i] * (LO ? s + sl : s);
    }
  }
}

// Gradient that the law of voxel (vx, vy) takes at point r, from the corner values
// (for J2 voxels the caller has already subtracted u^f_n from them).
template <typename T, int TETRA, bool LO>
__device__ __forceinline__ void law_grad(const ResParams<T>& P, bool j2, const T uh[3][8], const T ul[3][8], int r,
                                         int vx, int vy, int vz, T Gf[9], T Gt[9]) {
  point_grad<T, TETRA, LO>(uh, ul, r, P.wgrad, Gf);
  if (j2) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Gt[i] = Gf[i] + P.dGs[i];
    if (P.dquad) add_quad<T, TETRA>(P.hh, P.dQ, r, vx, vy, vz, Gt);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) Gt[i] = Gf[i] + P.Gs[i];
    if (P.quad) add_quad<T, TETRA>(P.hh, P.Qc, r, vx, vy, vz, Gt);
  }
  if (P.us[0]) {  // u* as a node field: the scheme's stencil on its corner values (its change
                  // since the commit for a J2 increment)
    T sh[3][8], sl[3][8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      int gx = vx + (o & 1), gy = vy + ((o >> 1) & 1), gz = vz + (o >> 2);
      if (P.periodic[0] && gx == P.n[0]) gx = 0;
      if (P.periodic[1] && gy == P.n[1]) gy = 0;
      if (P.periodic[2] && gz == P.n[2]) gz = 0;
      const long long at = gx + gy * P.nsy + gz * P.nsz;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T v = P.us[c][at];
        if (j2 && P.us_n[0]) v -= P.us_n[c][at];
        sh[c][o] = v;
        sl[c][o] = T(0);
      }
    }
    T Gu[9];
    point_grad<T, TETRA, false>(sh, sl, r, P.wgrad, Gu);
#pragma unroll
    for (int i = 0; i < 9; ++i) Gt[i] += Gu[i];
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  }
  return t;  // valid in thread 0
}

// ---- the residual as two passes over the grid ----------------------------------
// k_stress: one thread per voxel evaluates the gradient and the law at its
// point(s) and stores P (and tau for the test variant) in the voxel-point
// buffer vs[(r * NC + c) * nvox + voxel]: NC = 6 (11, 22, 33, 23, 13, 12) when
// every law gives a symmetric P, else 9 (c = 3 i + q); tau follows at c + NC.
// k_div: one thread per node gathers D = div P (and p = div tau) from the 8
// voxels around it.  Both run over 32 x 8 (x, y) tiles of one z plane with a
// fixed number of blocks, so the per-block FP64 partials (S_D from k_div, S_P
// from k_stress, same block index) have a bounded count.
constexpr int RTX = 32, RTY = 8, RBLOCKS = 2432;

// Tiles of RTX x RTY (x, y) positions of one z plane over the box [o, o + e).
struct TileIdx {
  int tx, ty, ntile;
  int ox, oy, oz;  // origin of the box
  int ex, ey, ez;  // extents of the box
  __device__ __forceinline__ void at(int t, int* x0, int* y0, int* z) const {
    *x0 = ox + (t % tx) * RTX;
    const int r = t / tx;
    *y0 = oy + (r % ty) * RTY;
    *z = oz + r / ty;
  }
};

static TileIdx make_tiles(int ox, int oy, int oz, int ex, int ey, int ez) {
  TileIdx ti;
  ti.ox = ox; ti.oy = oy; ti.oz = oz;
  ti.ex = ex; ti.ey = ey; ti.ez = ez;
  ti.tx = (ex + RTX - 1) / RTX;
  ti.ty = (ey + RTY - 1) / RTY;
  ti.ntile = (ex > 0 && ey > 0 && ez > 0) ? ti.tx * ti.ty * ez : 0;
  return ti;
}

// Nodes on non-periodic faces, each once: segment a holds the nodes with
// m_a in {0, n_a}, m_b interior for the non-periodic axes b < a.
struct FaceIdx {
  int count;
  int seg[3];     // nodes in segment a (0 for a periodic axis)
  int ext[3][3];  // extent along each axis in segment a
  int org[3][3];  // origin along each axis in segment a
  __device__ __forceinline__ bool at(int t, int n_face[3], int* m) const {
    for (int a = 0; a < 3; ++a) {
      if (t < seg[a]) {  // side 0's nodes, then side 1's (a warp stays on one face)
        const int half = seg[a] >> 1;
        const int side = t >= half;
        int r = side ? t - half : t;
        for (int b = 0; b < 3; ++b) {
          if (b == a) {
            m[b] = side ? n_face[a] : 0;
          } else {
            m[b] = org[a][b] + r % ext[a][b];
            r /= ext[a][b];
          }
        }
        return true;
      }
      t -= seg[a];
    }
    return false;
  }
};

__device__ __forceinline__ int sym_index(int i, int q) {
  if (i == q) return i;
  return 6 - i - q;  // (1,2) -> 3, (0,2) -> 4, (0,1) -> 5
}

template <typename T, int TETRA, bool WITH_P, bool LO, bool SYM, int SL>
__global__ void __launch_bounds__(RTX * RTY) k_stress(ResParams<T> P, TileIdx ti) {
  if (P.stop && *P.stop) return;
  constexpr bool J2 = (SL & 1) != 0;
  constexpr int NPP = TETRA ? 2 : 1;
  constexpr int NC = SYM ? 6 : 9;
  constexpr int NCT = WITH_P ? NC + 9 : NC;
  __shared__ double red[32];
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const long long nvox = (long long)n1 * n2 * n3;
  const int sy = (int)P.sy, sz = (int)P.sz, vy = (int)P.vy, vz_ = (int)P.vz;
  T sp = T(0);
  double SP = 0.0;
  int run = 0;
  for (int t = blockIdx.x; t < ti.ntile; t += gridDim.x) {
    int x0, y0, vz;
    ti.at(t, &x0, &y0, &vz);
    const int vx = x0 + (threadIdx.x % RTX), vy_ = y0 + (threadIdx.x / RTX);
    if (vx < n1 && vy_ < n2) {
      T uh[3][8], ul[3][8];
      int at[8], atn[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        int gx = vx + (o & 1), gy = vy_ + ((o >> 1) & 1), gz = vz + (o >> 2);
        if (P.periodic[0] && gx == n1) gx = 0;
        if (P.periodic[1] && gy == n2) gy = 0;
        if (P.periodic[2] && gz == n3) gz = 0;
        at[o] = gx + gy * sy + gz * sz;
        atn[o] = gx + gy * (int)P.nsy + gz * (int)P.nsz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          uh[c][o] = __ldg(P.u[c] + at[o]);
          ul[c][o] = LO ? __ldg(P.ulo[c] + at[o]) : T(0);
        }
      }
      const int v = vx + vy_ * vy + vz * vz_;
      const int ph = P.phase[v];
      const int law = __ldg(P.law_id + ph);
      const bool j2 = J2 && law == LAW_J2;
      const T* lc = P.law_c + (size_t)ph * LAWC;
      if (j2) {  // J2 takes the increment since the commit (u^f_n in the problem's own layout)
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          const int an = atn[o];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            uh[c][o] -= __ldg(P.un[c] + an);
            if (LO) ul[c][o] -= __ldg(P.unlo[c] + an);
            else if (P.unlo[c]) uh[c][o] -= __ldg(P.unlo[c] + an);  // a caller field without low part
          }
        }
      }
      T spv = T(0);
#pragma unroll
      for (int r = 0; r < NPP; ++r) {
        T Gf[9], Gt[9], Pp[9];
        law_grad<T, TETRA, LO>(P, j2, uh, ul, r, vx, vy_, vz, Gf, Gt);
        if (SL) point_law<T, SL>(P, law, lc, Gt, r, v, nvox, Pp, nullptr);
        else law_eval<T>(law, lc, Gt, Pp);
        T* base = P.vs + (size_t)(r * NCT) * nvox + v;
        if (SYM) {
          const T s6[6] = {Pp[0], Pp[4], Pp[8], Pp[5], Pp[2], Pp[1]};
#pragma unroll
          for (int c = 0; c < 6; ++c) base[(size_t)c * nvox] = s6[c];
        } else {
#pragma unroll
          for (int c = 0; c < 9; ++c) base[(size_t)c * nvox] = Pp[c];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) spv += Pp[c] * Pp[c];
        if (WITH_P) {
          if (j2) {  // tau takes grad u^f: add grad u^f_n back to the increment's gradient
            T nh[3][8], nl[3][8], Gn[9];
            for (int o = 0; o < 8; ++o) {
              int gx = vx + (o & 1), gy = vy_ + ((o >> 1) & 1), gz = vz + (o >> 2);
              if (P.periodic[0] && gx == n1) gx = 0;
              if (P.periodic[1] && gy == n2) gy = 0;
              if (P.periodic[2] && gz == n3) gz = 0;
              const int at = gx + gy * sy + gz * sz;
              for (int c = 0; c < 3; ++c) {
                nh[c][o] = P.un[c][at];
                nl[c][o] = LO ? P.unlo[c][at] : T(0);
              }
            }
            point_grad<T, TETRA, LO>(nh, nl, r, P.wgrad, Gn);
            for (int i = 0; i < 9; ++i) Gf[i] += Gn[i];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              T tq = P.two_mu0 * Gf[i * 3 + q] - Pp[i * 3 + q];
              if (i == q) tq += P.lam0 * (P.c0 ? Gf[0] + Gf[4] + Gf[8] : Gf[i * 3 + i]);
              base[(size_t)(NC + i * 3 + q) * nvox] = tq;
            }
        }
      }
      sp += spv;
    }
    if (++run == 16) {  // fold the run into FP64
      SP += (double)sp;
      sp = T(0);
      run = 0;
    }
  }
  SP += (double)sp;
  const double tot = block_sum(SP, red);
  if (threadIdx.x == 0) P.partial[2 * blockIdx.x + 1] = tot / NPP;
}

// Incremental variant of k_stress (J2 problems after their first commit): stores
// P - P_n, with P_n the stress at the commit (elastic laws: the law applied to the
// gradient increment; J2: j2_inc).  S_P still takes the full P.
template <typename T, int TETRA, bool LO, bool SYM>
__global__ void __launch_bounds__(RTX * RTY) k_stress_inc(ResParams<T> P, TileIdx ti) {
  if (P.stop && *P.stop) return;
  constexpr int NPP = TETRA ? 2 : 1;
  constexpr int NC = SYM ? 6 : 9;
  __shared__ double red[32];
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const long long nvox = (long long)n1 * n2 * n3;
  const int sy = (int)P.sy, sz = (int)P.sz, vy = (int)P.vy, vz_ = (int)P.vz;
  T sp = T(0);
  double SP = 0.0;
  int run = 0;
  for (int t = blockIdx.x; t < ti.ntile; t += gridDim.x) {
    int x0, y0, vz;
    ti.at(t, &x0, &y0, &vz);
    const int vx = x0 + (threadIdx.x % RTX), vy_ = y0 + (threadIdx.x / RTX);
    if (vx < n1 && vy_ < n2) {
      const int v = vx + vy_ * vy + vz * vz_;
      const int ph = P.phase[v];
      const int law = __ldg(P.law_id + ph);
      const bool j2 = law == LAW_J2;
      const T* lc = P.law_c + (size_t)ph * LAWC;
      T uh[3][8], ul[3][8];
      int at[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        int gx = vx + (o & 1), gy = vy_ + ((o >> 1) & 1), gz = vz + (o >> 2);
        if (P.periodic[0] && gx == n1) gx = 0;
        if (P.periodic[1] && gy == n2) gy = 0;
        if (P.periodic[2] && gz == n3) gz = 0;
        at[o] = gx + gy * sy + gz * sz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          uh[c][o] = __ldg(P.u[c] + at[o]);
          ul[c][o] = LO ? __ldg(P.ulo[c] + at[o]) : T(0);
        }
      }
      T spv = T(0);
      if (!j2) {  // |P|^2 of the elastic law on the total gradient
#pragma unroll
        for (int r = 0; r < NPP; ++r) {
          T Gf[9], Gt[9], Pp[9];
          law_grad<T, TETRA, LO>(P, false, uh, ul, r, vx, vy_, vz, Gf, Gt);
          law_eval<T>(law, lc, Gt, Pp);
#pragma unroll
          for (int c = 0; c < 9; ++c) spv += Pp[c] * Pp[c];
        }
      }
#pragma unroll
      for (int o = 0; o < 8; ++o)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          uh[c][o] -= __ldg(P.un[c] + at[o]);
          if (LO) ul[c][o] -= __ldg(P.unlo[c] + at[o]);
        }
#pragma unroll
      for (int r = 0; r < NPP; ++r) {
        T Gd[9], dG[9], dP[9];
        law_grad<T, TETRA, LO>(P, true, uh, ul, r, vx, vy_, vz, Gd, dG);
        if (j2) {
          const T* stp = P.state + (long long)(r * P.nst) * nvox + v;
          T st[7], Pf[9];
#pragma unroll
          for (int c = 0; c < 7; ++c) st[c] = stp[c * nvox];
          j2_inc<T>(lc, dG, st, dP, Pf, nullptr);
#pragma unroll
          for (int c = 0; c < 9; ++c) spv += Pf[c] * Pf[c];
        } else {
          law_eval<T>(law, lc, dG, dP);
        }
        T* base = P.vs + (size_t)(r * NC) * nvox + v;
        if (SYM) {
          const T s6[6] = {dP[0], dP[4], dP[8], dP[5], dP[2], dP[1]};
#pragma unroll
          for (int c = 0; c < 6; ++c) base[(size_t)c * nvox] = s6[c];
        } else {
#pragma unroll
          for (int c = 0; c < 9; ++c) base[(size_t)c * nvox] = dP[c];
        }
      }
      sp += spv;
    }
    if (++run == 16) {
      SP += (double)sp;
      sp = T(0);
      run = 0;
    }
  }
  SP += (double)sp;
  const double tot = block_sum(SP, red);
  if (threadIdx.x == 0) P.partial[2 * blockIdx.x + 1] = tot / NPP;
}

// General divergence at node (mx, my, mz), with the ghost rules on face nodes.
template <typename T, int TETRA, bool WITH_P, bool SYM>
__device__ __forceinline__ void node_div_general(const ResParams<T>& P, int mx, int my, int mz, T Dq[3], T pq[3],
                                                 int qmask = 7) {
  constexpr int NC = SYM ? 6 : 9;
  constexpr int NCT = WITH_P ? NC + 9 : NC;
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const int px = P.periodic[0], py = P.periodic[1], pz = P.periodic[2];
  const long long nvox = (long long)n1 * n2 * n3;
  auto corner = [&](int o, int i, int q, T* f) -> long long {
    const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
    int vx = mx + ox - 1, vy = my + oy - 1, vz = mz + oz - 1, cross = 0, sgn = 1;
    if (vx < 0 || vx >= n1) {
      if (px) vx = (vx + n1) % n1;
      else {
        sgn *= P.sgn[q][0][vx < 0 ? 0 : 1] * (i == 0 ? -1 : 1);
        vx = vx < 0 ? 0 : n1 - 1;
        ++cross;
      }
    }
    if (vy < 0 || vy >= n2) {
      if (py) vy = (vy + n2) % n2;
      else {
        sgn *= P.sgn[q][1][vy < 0 ? 0 : 1] * (i == 1 ? -1 : 1);
        vy = vy < 0 ? 0 : n2 - 1;
        ++cross;
      }
    }
    if (vz < 0 || vz >= n3) {
      if (pz) vz = (vz + n3) % n3;
      else {
        sgn *= P.sgn[q][2][vz < 0 ? 0 : 1] * (i == 2 ? -1 : 1);
        vz = vz < 0 ? 0 : n3 - 1;
        ++cross;
      }
    }
    int r = 0;
    if (TETRA) {
      r = ((ox + oy + oz) & 1) ? 0 : 1;  // odd corner -> T1 point (div_T2), even -> T2 (div_T1)
      if (cross & 1) r ^= 1;
    }
    *f = T(sgn);
    return (long long)(r * NCT) * nvox + vx + vy * P.vy + (long long)vz * P.vz;
  };
  // component outermost, the three directions unrolled: a component's 24 gathers are
  // independent and in flight together (the sums over i keep their order)
  for (int q = 0; q < 3; ++q) {
    if (!((qmask >> q) & 1)) continue;  // a component without a dof at this node stays zero
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int c = SYM ? sym_index(i, q) : i * 3 + q;
      T s = T(0), st = T(0);
      // imposed stress of a traction on the face normal to i that this node lies on: every
      // pair along i has its ghost corner there (Sec. 2.2, P* = 2 t at the mirror centres)
      // side 0: - (2 (-1) t) at corner o; side 1: + (2 t) at corner o1 -- both add 2 t
      int side = -1;
      if (P.traction && !P.periodic[i]) {
        const int m_i = i == 0 ? mx : (i == 1 ? my : mz);
        if (m_i == 0 && P.sgn[q][i][0] > 0) side = 0;
        else if (m_i == P.n[i] && P.sgn[q][i][1] > 0) side = 1;
      }
      const T* tfc = side >= 0 ? P.tface[i][side] : nullptr;
      const T* tfn = side >= 0 ? P.tface_n[i][side] : nullptr;
      const T ps_u = side >= 0 ? T(2) * P.tr[i][side][q] : T(0);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        if ((o >> i) & 1) continue;
        const int o1 = o | (1 << i);
        T f0, f1;
        const long long a0 = corner(o, i, q, &f0);
        const long long a1 = corner(o1, i, q, &f1);
        T ps = ps_u;
        if (tfc || tfn) {  // the field at the face voxel that this pair's ghost corner mirrors
          const int b = i == 0 ? 1 : 0, cc = i == 2 ? 1 : 2;
          const int mb = b == 0 ? mx : my, mc = cc == 1 ? my : mz;
          const int nb = P.n[b], nc = P.n[cc];
          int vb = mb + ((o >> b) & 1) - 1, vc = mc + ((o >> cc) & 1) - 1;
          if (vb < 0) vb = P.periodic[b] ? nb - 1 : 0;
          if (vb >= nb) vb = P.periodic[b] ? 0 : nb - 1;
          if (vc < 0) vc = P.periodic[cc] ? nc - 1 : 0;
          if (vc >= nc) vc = P.periodic[cc] ? 0 : nc - 1;
          const long long at = (long long)q * nb * nc + vb + (long long)nb * vc;
          if (tfc) ps += T(2) * tfc[at];
          if (tfn) ps -= T(2) * tfn[at];
        }
        s += f1 * P.vs[a1 + c * nvox] - f0 * P.vs[a0 + c * nvox] + ps;
        if (WITH_P) st += f1 * P.vs[a1 + (NC + i * 3 + q) * nvox] - f0 * P.vs[a0 + (NC + i * 3 + q) * nvox];
      }
      Dq[q] += P.wdiv[i] * s;
      if (WITH_P) pq[q] += P.wdiv[i] * st;
    }
  }
}

template <typename T, bool WITH_P, bool INC>
__device__ __forceinline__ T store_node(const ResParams<T>& P, int mx, int my, int mz, const T Dq[3], const T pq[3]) {
  const int off = mx + my * (int)P.sy + mz * (int)P.sz;
  T sdn = T(0);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool dof = mx >= P.lo[q][0] && mx < P.hi[q][0] && my >= P.lo[q][1] && my < P.hi[q][1] &&
                     mz >= P.lo[q][2] && mz < P.hi[q][2];
    const T d = INC ? Dq[q] + __ldg(P.Dn[q] + off) : Dq[q];
    P.D[q][off] = dof ? d : T(0);
    if (WITH_P) P.p[q][off] = dof ? pq[q] : T(0);
    if (dof) sdn += d * d;
  }
  return sdn;
}

// Interior nodes: all 8 neighbouring voxels exist (or wrap); plain differences.
template <typename T, int TETRA, bool WITH_P, bool SYM, bool INC>
__global__ void __launch_bounds__(RTX * RTY) k_div(ResParams<T> P, TileIdx ti, FaceIdx fi) {
  if (P.stop && *P.stop) return;
  constexpr int NC = SYM ? 6 : 9;
  constexpr int NCT = WITH_P ? NC + 9 : NC;
  __shared__ double red[32];
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const long long nvox = (long long)n1 * n2 * n3;
  const int vy = (int)P.vy, vz_ = (int)P.vz;
  T sd = T(0);
  double SD = 0.0;
  int run = 0;
  for (int t = blockIdx.x; t < ti.ntile; t += gridDim.x) {
    int x0, y0, mz;
    ti.at(t, &x0, &y0, &mz);
    const int mx = x0 + (threadIdx.x % RTX), my = y0 + (threadIdx.x / RTX);
    if (mx < ti.ox + ti.ex && my < ti.oy + ti.ey) {
      T Dq[3] = {T(0), T(0), T(0)}, pq[3] = {T(0), T(0), T(0)};
      int vidx[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        int vx = mx + (o & 1) - 1, vyy = my + ((o >> 1) & 1) - 1, vz = mz + (o >> 2) - 1;
        if (vx < 0) vx += n1;
        if (vyy < 0) vyy += n2;
        if (vz < 0) vz += n3;
        vidx[o] = vx + vyy * vy + vz * vz_;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int c = SYM ? sym_index(i, q) : i * 3 + q;
          const T* b0 = P.vs + (size_t)c * nvox;                  // T1 point
          const T* b1 = P.vs + (size_t)(NCT + c) * nvox;          // T2 point
          const T* t0 = P.vs + (size_t)(NC + i * 3 + q) * nvox;   // tau, T1
          const T* t1 = P.vs + (size_t)(NCT + NC + i * 3 + q) * nvox;
          T s = T(0), st = T(0);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            if ((o >> i) & 1) continue;
            const int o1 = o | (1 << i);
            // odd-parity corner -> T1 point, even -> T2 point (HEX1: the single point)
            const bool odd0 = (((o & 1) + ((o >> 1) & 1) + (o >> 2)) & 1) != 0;
            const bool odd1 = !odd0;
            const T* p0 = (!TETRA || odd0) ? b0 : b1;
            const T* p1 = (!TETRA || odd1) ? b0 : b1;
            s += __ldg(p1 + vidx[o1]) - __ldg(p0 + vidx[o]);
            if (WITH_P) {
              const T* q0 = (!TETRA || odd0) ? t0 : t1;
              const T* q1 = (!TETRA || odd1) ? t0 : t1;
              st += __ldg(q1 + vidx[o1]) - __ldg(q0 + vidx[o]);
            }
          }
          Dq[q] += P.wdiv[i] * s;
          if (WITH_P) pq[q] += P.wdiv[i] * st;
        }
      }
      sd += store_node<T, WITH_P, INC>(P, mx, my, mz, Dq, pq);
    }
    if (++run == 16) {
      SD += (double)sd;
      sd = T(0);
      run = 0;
    }
  }
  // face nodes, each once, with the ghost rules
  int nface[3] = {n1, n2, n3};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < fi.count; t += gridDim.x * blockDim.x) {
    int m[3];
    if (!fi.at(t, nface, m)) continue;
    T Dq[3] = {T(0), T(0), T(0)}, pq[3] = {T(0), T(0), T(0)};
    node_div_general<T, TETRA, WITH_P, SYM>(P, m[0], m[1], m[2], Dq, pq);
    SD += (double)store_node<T, WITH_P, INC>(P, m[0], m[1], m[2], Dq, pq);
  }
  SD += (double)sd;
  const double tot = block_sum(SD, red);
  if (threadIdx.x == 0) P.partial[2 * blockIdx.x] = tot;
}

static TileIdx voxel_tiles(const int n[3]) { return make_tiles(0, 0, 0, n[0], n[1], n[2]); }

template <typename T>
static void interior_and_faces(const ResParams<T>& P, TileIdx* ti, FaceIdx* fi) {
  int o[3], e[3];
  for (int a = 0; a < 3; ++a) {
    o[a] = P.periodic[a] ? 0 : 1;              // interior node range [1, n) on a non-periodic axis
    e[a] = P.periodic[a] ? P.N[a] : P.n[a] - 1;
  }
  *ti = make_tiles(o[0], o[1], o[2], e[0], e[1], e[2]);
  fi->count = 0;
  for (int a = 0; a < 3; ++a) {
    fi->seg[a] = 0;
    for (int b = 0; b < 3; ++b) {
      fi->org[a][b] = 0;
      fi->ext[a][b] = 1;
    }
    if (P.periodic[a]) continue;
    int cnt = 2;
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      if (b < a && !P.periodic[b]) {
        fi->org[a][b] = 1;
        fi->ext[a][b] = P.n[b] - 1;
      } else {
        fi->org[a][b] = 0;
        fi->ext[a][b] = P.N[b];
      }
      cnt *= fi->ext[a][b];
    }
    fi->seg[a] = cnt;
    fi->count += cnt;
  }
}

// ---- the residual as one pass (small-strain elastic laws) -----------------------
// k_residual_fused: a block marches a tile of FX x FY voxels (x, y) through a chunk of z
// planes.  Per z step it (1) stores the next node plane of u^f (FX+1 x FY+1 nodes, hi and
// lo parts) in shared memory, then, after the step's one barrier, (2) forms D at the node
// plane below the previous voxel layer, from the 8 voxels around each node, as the same sums
// of neighbour differences as k_div (Remark 1), and (3) evaluates the gradient and the law of
// its voxel layer from the two node planes around it (the lower plane's corners stay in
// registers from the previous step), keeping the voxel-point stresses in shared memory: a
// ring of three layers, so that the layer being written is never one that (2) reads.  The block's
// voxel tile overlaps its neighbours' by one voxel in x and y so that the (FX-1) x (FY-1)
// nodes it owns see all their voxels; the stresses never leave the SM.  Nodes on
// non-periodic faces take the ghost rules in k_face_div, which reads the stresses of the
// boundary voxel layers that this kernel stores to the voxel-point buffer.
constexpr int FX = 32, FNX = FX + 1;  // voxel tile width in x (one warp); tile height FY is 8 or 16

// u^f at a node in shared memory: (hi, lo) in FP32, the value in FP64
template <typename T, bool LO> struct NodeV { using t = T; };
template <> struct NodeV<float, true> { using t = float2; };
__device__ __forceinline__ float nv_hi(float2 v) { return v.x; }
__device__ __forceinline__ float nv_lo(float2 v) { return v.y; }
__device__ __forceinline__ float nv_hi(float v) { return v; }
__device__ __forceinline__ float nv_lo(float) { return 0.f; }
__device__ __forceinline__ double nv_hi(double v) { return v; }
__device__ __forceinline__ double nv_lo(double) { return 0.0; }

// Work decomposition of the fused residual: per axis, the interior node range [a0, a1)
// (every node on a periodic axis, [1, n) on a non-periodic one), tiles of FX-1 (x) and
// FY-1 (y) nodes, chunks of zc node planes in z.
struct FusedGeom {
  int fy;  // voxel tile height (8 or 16)
  int a0[3], a1[3];
  int ntx, nty, nzc, zc;
  int items;
  int faces;  // 1 if some axis is non-periodic: boundary voxel layers go to the stress buffer
  int fdof[3];  // the faces normal to axis a hold a dof of some component: their voxel layers
                // go to the stress buffer (the face kernel reads no other)
};

template <typename T>
static FusedGeom fused_geom(const ResParams<T>& P) {
  FusedGeom g;
  g.fy = P.fused_fy == 16 ? 16 : 8;
  const int FY = g.fy;
  for (int a = 0; a < 3; ++a) {
    g.a0[a] = P.periodic[a] ? 0 : 1;
    g.a1[a] = P.n[a];
  }
  g.ntx = (g.a1[0] - g.a0[0] + FX - 2) / (FX - 1);
  g.nty = (g.a1[1] - g.a0[1] + FY - 2) / (FY - 1);
  const int nz = g.a1[2] - g.a0[2];
  const long long cols = (long long)g.ntx * g.nty;
  // chunks of at least 16 planes, few enough that the blocks stay below ~4000
  int zc = (int)((cols * nz + 3999) / 4000);
  zc = zc < 16 ? 16 : zc;
  zc = zc > nz ? nz : zc;
  g.zc = zc > 0 ? zc : 1;
  g.nzc = nz > 0 ? (nz + g.zc - 1) / g.zc : 0;
  g.items = (int)(cols * g.nzc);
  g.faces = !(P.periodic[0] && P.periodic[1] && P.periodic[2]);
  for (int a = 0; a < 3; ++a) {
    g.fdof[a] = 0;
    if (P.periodic[a]) continue;
    for (int q = 0; q < 3; ++q)
      if (P.lo[q][a] == 0 || P.hi[q][a] > P.n[a]) g.fdof[a] = 1;
  }
  return g;
}

// The first 24 coefficients of a phase's law row (isotropic: lambda, mu; cubic: the upper
// triangle of the rotated Mandel stiffness, 21 entries), loaded together as vectors.
template <typename T>
__device__ __forceinline__ void load_law24(const T* __restrict__ lc, T c[24]) {
  if constexpr (sizeof(T) == 4) {
    const float4* v = reinterpret_cast<const float4*>(lc);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 a = __ldg(v + i);
      c[4 * i] = a.x; c[4 * i + 1] = a.y; c[4 * i + 2] = a.z; c[4 * i + 3] = a.w;
    }
  } else {
    const double2* v = reinterpret_cast<const double2*>(lc);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const double2 a = __ldg(v + i);
      c[2 * i] = a.x; c[2 * i + 1] = a.y;
    }
  }
}

// Small-strain elastic law from coefficients in registers: P as (11, 22, 33, 23, 13, 12).
template <typename T>
__device__ __forceinline__ void elastic_reg(int law, const T c[24], const T G[9], T s[6]) {
  const T e00 = G[0], e11 = G[4], e22 = G[8];
  const T e12 = T(0.5) * (G[5] + G[7]), e02 = T(0.5) * (G[2] + G[6]), e01 = T(0.5) * (G[1] + G[3]);
  if (law == LAW_CUBIC) {
    const T r2 = T(1.41421356237309504880), ir2 = T(0.70710678118654752440);
    const T em[6] = {e00, e11, e22, r2 * e12, r2 * e02, r2 * e01};
    T sm[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    int k = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) {
        const T v = c[k++];
        sm[a] += v * em[b];
        if (b != a) sm[b] += v * em[a];
      }
    s[0] = sm[0]; s[1] = sm[1]; s[2] = sm[2];
    s[3] = ir2 * sm[3]; s[4] = ir2 * sm[4]; s[5] = ir2 * sm[5];
  } else {  // isotropic
    const T mu2 = T(2) * c[1], tr = c[0] * (e00 + e11 + e22);
    s[0] = tr + mu2 * e00; s[1] = tr + mu2 * e11; s[2] = tr + mu2 * e22;
    s[3] = mu2 * e12; s[4] = mu2 * e02; s[5] = mu2 * e01;
  }
}

// Gradient at point r from the corner values of the lower (L, corners o < 4) and upper
// (U, corners o >= 4) node planes, as point_grad forms it.  The FP32 variant takes (hi, lo)
// pairs and uses packed FP32x2 arithmetic (one instruction per pair) with the same
// differences, sums and rounding.
template <int TETRA>
__device__ __forceinline__ void grad_lu_f2(const float2 L[3][4], const float2 U[3][4], int r, const float* wg,
                                           float G[9]) {
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int mask = TETRA ? ((1 << i) | (1 << ((i + 1) % 3))) : (1 << i);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        if ((o >> i) & 1) continue;
        const int par = ((o & 1) + ((o >> 1) & 1) + ((o >> 2) & 1)) & 1;
        if (TETRA && ((r == 0) != (par == 0))) continue;
        const int o2 = o ^ mask;
        const float2 a = o < 4 ? L[q][o] : U[q][o - 4];
        const float2 b = o2 < 4 ? L[q][o2] : U[q][o2 - 4];
        s = __fadd2_rn(s, __ffma2_rn(a, m1, b));  // + (u(o ^ mask) - u(o))
      }
      G[i * 3 + q] = wg[i] * (s.x + s.y);
    }
  }
}

template <typename T, int TETRA>
__device__ __forceinline__ void grad_lu(const T L[3][4], const T U[3][4], int r, const T* wg, T G[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int mask = TETRA ? ((1 << i) | (1 << ((i + 1) % 3))) : (1 << i);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T s = T(0);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        if ((o >> i) & 1) continue;
        const int par = ((o & 1) + ((o >> 1) & 1) + ((o >> 2) & 1)) & 1;
        if (TETRA && ((r == 0) != (par == 0))) continue;
        const int o2 = o ^ mask;
        s += (o2 < 4 ? L[q][o2] : U[q][o2 - 4]) - (o < 4 ? L[q][o] : U[q][o - 4]);
      }
      G[i * 3 + q] = wg[i] * s;
    }
  }
}

// Small-strain elastic law with the phase's full Mandel stiffness (9 blocks of 2 x 2, see
// ResParams::law_m) and packed FP32x2 products: P as (11, 22, 33, 23, 13, 12).
__device__ __forceinline__ void elastic_f2(const float4* __restrict__ M4, const float G[9], float s[6]) {
  const float r2 = 1.41421356237309504880f, ir2 = 0.70710678118654752440f;
  const float em[6] = {G[0], G[4], G[8], r2 * (0.5f * (G[5] + G[7])), r2 * (0.5f * (G[2] + G[6])),
                       r2 * (0.5f * (G[1] + G[3]))};
  float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
  for (int bp = 0; bp < 3; ++bp) {
    const float2 e0 = make_float2(em[2 * bp], em[2 * bp]), e1 = make_float2(em[2 * bp + 1], em[2 * bp + 1]);
#pragma unroll
    for (int rp = 0; rp < 3; ++rp) {
      const float4 c = __ldg(M4 + 3 * bp + rp);
      acc[rp] = __ffma2_rn(make_float2(c.x, c.y), e0, acc[rp]);
      acc[rp] = __ffma2_rn(make_float2(c.z, c.w), e1, acc[rp]);
    }
  }
  s[0] = acc[0].x;
  s[1] = acc[0].y;
  s[2] = acc[1].x;
  s[3] = ir2 * acc[1].y;
  s[4] = ir2 * acc[2].x;
  s[5] = ir2 * acc[2].y;
}

template <int V> struct Par { static constexpr int value = V; };

template <typename T, int TETRA, bool LO, int FY>
__global__ void __launch_bounds__(FX * FY, 16 / FY) k_residual_fused(ResParams<T> P, FusedGeom g) {
  if (P.stop && *P.stop) return;
  constexpr int FNY = FY + 1, FTHREADS = FX * FY;
  using NV = typename NodeV<T, LO>::t;
  using T2 = typename V2<T>::t;
  constexpr int NPP = TETRA ? 2 : 1;
  constexpr int PL = FNY * FNX;    // one component of one node plane
  constexpr int SL = FY * FX;      // one stress pair of one point of one voxel layer
  extern __shared__ __align__(16) unsigned char fsm[];
  NV* su = reinterpret_cast<NV*>(fsm);                      // [2][3][FNY][FNX] node planes
  T2* ss = reinterpret_cast<T2*>(su + 2 * 3 * PL);          // [3][NPP][3][FY][FX] stress pairs
  __shared__ double red[32];

  const int tx = threadIdx.x % FX, ty = threadIdx.x / FX;
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const int N1 = P.N[0], N2 = P.N[1], N3 = P.N[2];
  const long long nvox = (long long)n1 * n2 * n3;
  const long long sy = P.sy, sz = P.sz;
  const int item = blockIdx.x;
  const int ix = item % g.ntx, iy = (item / g.ntx) % g.nty, iz = item / (g.ntx * g.nty);
  const int X0 = g.a0[0] + ix * (FX - 1), Y0 = g.a0[1] + iy * (FY - 1);
  const int Z0 = g.a0[2] + iz * g.zc, Z1 = min(Z0 + g.zc, g.a1[2]);
  const int Xend = min(X0 + FX - 1, g.a1[0]), Yend = min(Y0 + FY - 1, g.a1[1]);

  // this thread's voxel column (x, y) and node (x, y)
  int vx = X0 - 1 + tx, vy = Y0 - 1 + ty;
  const bool vin = (vx >= 0 || P.periodic[0]) && (vx < n1) && (vy >= 0 || P.periodic[1]) && (vy < n2);
  if (vx < 0) vx += n1;
  if (vy < 0) vy += n2;
  const int mx = X0 - 1 + tx, my = Y0 - 1 + ty;
  const bool node_out = tx >= 1 && ty >= 1 && mx < Xend && my < Yend;
  // voxels this block counts in S_P and stores for the face kernel: the core [X0, Xend) of
  // the tile, plus voxel 0 for the first tile of a non-periodic axis
  const int ox_lo = X0 - ((ix == 0 && !P.periodic[0]) ? 1 : 0);
  const int oy_lo = Y0 - ((iy == 0 && !P.periodic[1]) ? 1 : 0);
  const bool own_xy = vin && mx >= ox_lo && mx < Xend && my >= oy_lo && my < Yend;
  const bool xy_face = (g.fdof[0] && (vx == 0 || vx == n1 - 1)) || (g.fdof[1] && (vy == 0 || vy == n2 - 1));
  const int phase_xy = vx + vy * (int)P.vy;
  const int own_z0 = Z0 - (iz == 0 && !P.periodic[2] ? 1 : 0);
  const long long node_xy = node_out ? mx + my * sy : 0;

  // the node slots this thread loads per plane: FNX x FNY nodes over FTHREADS threads
  long long gxy[2];
  bool gok[2];
#pragma unroll
  for (int sl = 0; sl < 2; ++sl) {
    const int idx = threadIdx.x + sl * FTHREADS;
    gok[sl] = idx < PL;
    int x = X0 - 1 + idx % FNX, y = Y0 - 1 + idx / FNX;
    if (x < 0) x += N1;  // only periodic axes reach -1 (non-periodic tiles start at 1)
    if (y < 0) y += N2;
    if (x >= N1) x -= N1;
    if (y >= N2) y -= N2;
    gxy[sl] = gok[sl] ? x + y * sy : 0;
  }
  NV pre[2][3];
  auto fetch_plane = [&](int z) {
    if (z < 0) z += N3;
    if (z >= N3) z -= N3;
    const long long zo = z * sz;
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      if (gok[sl]) {
        const long long at = gxy[sl] + zo;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if constexpr (LO) pre[sl][c] = make_float2(__ldg(P.u[c] + at), __ldg(P.ulo[c] + at));
          else pre[sl][c] = __ldg(P.u[c] + at);
        }
      }
    }
  };
  auto store_plane = [&](auto par) {
    constexpr int b = decltype(par)::value;
#pragma unroll
    for (int sl = 0; sl < 2; ++sl)
      if (gok[sl])
#pragma unroll
        for (int c = 0; c < 3; ++c) su[(b * 3 + c) * PL + threadIdx.x + sl * FTHREADS] = pre[sl][c];
  };
  NV* const su_me = su + ty * FNX + tx;
  auto read4 = [&](auto par, NV (&cv)[3][4]) {
    constexpr int b = decltype(par)::value;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) cv[c][k] = su_me[(b * 3 + c) * PL + (k >> 1) * FNX + (k & 1)];
  };

  T sp = T(0), sd = T(0);
  double SP = 0.0, SD = 0.0;
  int run = 0;

  // phase of this thread's voxel in layer vz (prefetched one layer ahead)
  auto phase_at = [&](int vz) -> int {
    if (!vin) return 0;
    if (vz < 0) vz += n3;
    if (vz >= n3) return 0;
    return P.phase[phase_xy + (long long)vz * P.vz];
  };
  T2* const ss_me = ss + ty * FX + tx;
  // voxel layer vz from the corner planes L (lower) and U (upper): stresses into stress
  // buffer b, S_P, boundary layers to the stress buffer of the face kernel
  auto voxel_layer = [&](int b, int vz, int ph, const NV (&L)[3][4], const NV (&U)[3][4]) {
    const bool zin = vz >= 0 && vz < n3;
    const int vzz = vz < 0 ? vz + n3 : vz;
    T Ps[NPP][6];
#pragma unroll
    for (int r = 0; r < NPP; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) Ps[r][c] = T(0);
    if (vin && (zin || P.periodic[2])) {
      if constexpr (LO) {  // FP32 hi + lo fields: packed FP32x2 gradient and law
        const float4* M4 = reinterpret_cast<const float4*>(P.law_m + (size_t)ph * 36);
#pragma unroll
        for (int r = 0; r < NPP; ++r) {
          float Gf[9], Gt[9];
          grad_lu_f2<TETRA>(L, U, r, P.wgrad, Gf);
#pragma unroll
          for (int i = 0; i < 9; ++i) Gt[i] = Gf[i] + P.Gs[i];
          if (P.quad) add_quad<T, TETRA>(P.hh, P.Qc, r, vx, vy, vzz, Gt);
          elastic_f2(M4, Gt, Ps[r]);
        }
      } else {
        const int law = __ldg(P.law_id + ph);
        T lc[24];
        load_law24<T>(P.law_c + (size_t)ph * LAWC, lc);
#pragma unroll
        for (int r = 0; r < NPP; ++r) {
          T Gf[9], Gt[9];
          grad_lu<T, TETRA>(L, U, r, P.wgrad, Gf);
#pragma unroll
          for (int i = 0; i < 9; ++i) Gt[i] = Gf[i] + P.Gs[i];
          if (P.quad) add_quad<T, TETRA>(P.hh, P.Qc, r, vx, vy, vzz, Gt);
          elastic_reg<T>(law, lc, Gt, Ps[r]);
        }
      }
      if (own_xy && vz >= own_z0 && vz < Z1) {
        T spv = T(0);
#pragma unroll
        for (int r = 0; r < NPP; ++r)
          spv += Ps[r][0] * Ps[r][0] + Ps[r][1] * Ps[r][1] + Ps[r][2] * Ps[r][2] +
                 T(2) * (Ps[r][3] * Ps[r][3] + Ps[r][4] * Ps[r][4] + Ps[r][5] * Ps[r][5]);
        sp += spv;
        if (g.faces && (xy_face || (g.fdof[2] && (vzz == 0 || vzz == n3 - 1)))) {
          const long long v = phase_xy + (long long)vzz * P.vz;
#pragma unroll
          for (int r = 0; r < NPP; ++r) {
            T* base = P.vs + (size_t)(r * 6) * nvox + v;
#pragma unroll
            for (int c = 0; c < 6; ++c) base[c * nvox] = Ps[r][c];
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NPP; ++r) {
      T2 a0, a1, a2;
      a0.x = Ps[r][0]; a0.y = Ps[r][1];  // 11, 22
      a1.x = Ps[r][2]; a1.y = Ps[r][3];  // 33, 23
      a2.x = Ps[r][4]; a2.y = Ps[r][5];  // 13, 12
      ss_me[((b * NPP + r) * 3 + 0) * SL] = a0;
      ss_me[((b * NPP + r) * 3 + 1) * SL] = a1;
      ss_me[((b * NPP + r) * 3 + 2) * SL] = a2;
    }
  };
  const T2* const ss_nb = ss + (ty > 0 ? ty - 1 : 0) * FX + (tx > 0 ? tx - 1 : 0);
  // D at node plane z from the voxel layers below (stress slot bl) and above (bu)
  auto node_div = [&](int bl, int bu, int z) {
    T val[8][6];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
      const int r = TETRA ? ((((ox + oy + oz) & 1) != 0) ? 0 : 1) : 0;
      const int b = oz ? bu : bl;
      const T2* p = ss_nb + ((b * NPP + r) * 3) * SL + oy * FX + ox;
      const T2 a0 = p[0], a1 = p[SL], a2 = p[2 * SL];
      val[o][0] = a0.x; val[o][1] = a0.y; val[o][2] = a1.x;
      val[o][3] = a1.y; val[o][4] = a2.x; val[o][5] = a2.y;
    }
    T Dq[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int c = sym_index(i, q);
        T s = T(0);
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          if ((o >> i) & 1) continue;
          s += val[o | (1 << i)][c] - val[o][c];
        }
        Dq[q] += P.wdiv[i] * s;
      }
    const long long off = node_xy + z * sz;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      P.D[q][off] = Dq[q];  // interior nodes transform every component (Table 1 ranges)
      sd += Dq[q] * Dq[q];
    }
  };

  // one z step: node plane z + 1 into node buffer B; after the barrier, D at node plane z - 1
  // (voxel layers z - 2 and z - 1, published by this barrier) and voxel layer z from (Lo, Up)
  // into stress slot sz_cur.  Voxel layer l sits in slot (l - Z0 + 1) % 3: it is written in
  // step l and read in steps l + 1 and l + 2, and its slot is written again in step l + 3,
  // after the barrier that ends step l + 2.
  NV cA[3][4], cB[3][4];
  int ph_next = 0;
  int s_lo = 0, s_mid = 0, s_cur = 1;  // slots of layers z - 2, z - 1 and z
  auto step = [&](auto par, int z, const NV (&Lo)[3][4], NV (&Up)[3][4]) {
    constexpr int B = decltype(par)::value;
    store_plane(Par<B>{});
    __syncthreads();
    if (z + 2 <= Z1) fetch_plane(z + 2);  // in flight during this layer
    const int ph = ph_next;
    if (z + 1 < Z1) ph_next = phase_at(z + 1);
    if (z > Z0 && node_out) node_div(s_lo, s_mid, z - 1);
    read4(Par<B>{}, Up);
    voxel_layer(s_cur, z, ph, Lo, Up);
    s_lo = s_mid;
    s_mid = s_cur;
    s_cur = s_cur == 2 ? 0 : s_cur + 1;
    if (++run == 16) {
      SP += (double)sp;
      SD += (double)sd;
      sp = sd = T(0);
      run = 0;
    }
  };

  // prologue: node planes Z0 - 1 (buffer 0) and Z0 (buffer 1), voxel layer Z0 - 1 (slot 0)
  ph_next = phase_at(Z0 - 1);
  fetch_plane(Z0 - 1);
  store_plane(Par<0>{});
  fetch_plane(Z0);
  store_plane(Par<1>{});
  __syncthreads();
  read4(Par<0>{}, cB);
  read4(Par<1>{}, cA);
  __syncthreads();  // buffer 0 is refilled by the first step
  {
    const int ph = ph_next;
    ph_next = phase_at(Z0);
    voxel_layer(0, Z0 - 1, ph, cB, cA);
    s_mid = 0;
  }
  if (Z0 + 1 <= Z1) fetch_plane(Z0 + 1);
  // steps alternate node buffers; the corners of plane z stay in registers (cA, cB in turn)
  for (int z = Z0; z < Z1; z += 2) {
    step(Par<0>{}, z, cA, cB);
    if (z + 1 < Z1) step(Par<1>{}, z + 1, cB, cA);
  }
  // the last node plane: voxel layers Z1 - 2 and Z1 - 1
  __syncthreads();
  if (Z1 > Z0 && node_out) node_div(s_lo, s_mid, Z1 - 1);
  SP += (double)sp;
  SD += (double)sd;
  const double tsp = block_sum(SP, red);
  const double tsd = block_sum(SD, red);
  if (threadIdx.x == 0) {
    P.partial[2 * blockIdx.x] = tsd;
    P.partial[2 * blockIdx.x + 1] = tsp / NPP;
  }
}

// Nodes on non-periodic faces (each once), with the ghost rules, from the boundary voxel
// layers that k_residual_fused stored; one S_D partial per block (S_P slot zero).  A thread
// takes one component of one node (component-major, so that a warp walks one face): the
// gathers of a node's three components run in parallel, and a component without a dof there
// (every component of a fully Dirichlet face) writes its zero without any gather.
template <typename T, int TETRA>
__global__ void __launch_bounds__(256, 2) k_face_div(ResParams<T> P, FaceIdx fi) {
  if (P.stop && *P.stop) return;
  __shared__ double red[32];
  double SD = 0.0;
  int nface[3] = {P.n[0], P.n[1], P.n[2]};
  const long long total = 3LL * fi.count;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / fi.count), k = (int)(t - (long long)q * fi.count);
    int m[3];
    if (!fi.at(k, nface, m)) continue;
    const bool dof = m[0] >= P.lo[q][0] && m[0] < P.hi[q][0] && m[1] >= P.lo[q][1] && m[1] < P.hi[q][1] &&
                     m[2] >= P.lo[q][2] && m[2] < P.hi[q][2];
    T Dq[3] = {T(0), T(0), T(0)}, pq[3] = {T(0), T(0), T(0)};
    if (dof) node_div_general<T, TETRA, false, true>(P, m[0], m[1], m[2], Dq, pq, 1 << q);
    const long long off = m[0] + m[1] * P.sy + m[2] * P.sz;
    P.D[q][off] = dof ? Dq[q] : T(0);
    if (dof) SD += (double)(Dq[q] * Dq[q]);
  }
  const double tot = block_sum(SD, red);
  if (threadIdx.x == 0) {
    P.partial[2 * blockIdx.x] = tot;
    P.partial[2 * blockIdx.x + 1] = 0.0;
  }
}

constexpr int kFaceBlocks = 152 * 8;  // a few node components per thread at 256^3 (each a chain of gathers)

template <typename T>
static size_t fused_smem(int tetra, int fy) {
  using NVs = typename NodeV<T, true>::t;  // same size as the FP64 node value
  return (size_t)2 * 3 * (fy + 1) * FNX * sizeof(NVs) + (size_t)3 * (tetra ? 2 : 1) * 3 * fy * FX * 2 * sizeof(T);
}

template <typename T, int TETRA, bool LO, int FY>
static cudaError_t launch_fused_kernel(const ResParams<T>& P, const FusedGeom& g, cudaStream_t s) {
  auto kern = k_residual_fused<T, TETRA, LO, FY>;
  const size_t smem = fused_smem<T>(TETRA, FY);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) kern<<<g.items, FX * FY, smem, s>>>(P, g);
  return e;
}

// The fused path serves the solver's residual for problems whose every law is a
// small-strain elastic one (isotropic or cubic: symmetric P, no internal variables), in the
// plain (non-incremental) form without the test outputs.
template <typename T>
static bool fused_ok(const ResParams<T>& P, bool with_p) {
  return !with_p && !P.inc && P.nst == 0 && P.sym && P.state == nullptr && !P.two_pass && P.us[0] == nullptr;
}

template <typename T>
static int fused_blocks(const ResParams<T>& P) {
  const FusedGeom g = fused_geom(P);
  return g.items + (g.faces ? kFaceBlocks : 0);
}

template <typename T, int TETRA>
static cudaError_t launch_fused_t(const ResParams<T>& P, cudaStream_t s, int* blocks_out) {
  const FusedGeom g = fused_geom(P);
  const bool lo = P.ulo[0] != nullptr;
  if (g.items > 0) {
    cudaError_t e = cudaSuccess;
    if (lo) {
      if constexpr (sizeof(T) == 4) {  // FP32 with a low part (the solver's fields)
        e = g.fy == 16 ? launch_fused_kernel<T, TETRA, true, 16>(P, g, s) : launch_fused_kernel<T, TETRA, true, 8>(P, g, s);
      } else {
        return cudaErrorInvalidValue;  // FP64 fields carry no low part
      }
    } else {
      e = g.fy == 16 ? launch_fused_kernel<T, TETRA, false, 16>(P, g, s) : launch_fused_kernel<T, TETRA, false, 8>(P, g, s);
    }
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  int blocks = g.items;
  if (g.faces) {
    TileIdx tn;
    FaceIdx fi;
    interior_and_faces<T>(P, &tn, &fi);
    ResParams<T> Pf = P;
    Pf.partial = P.partial + 2 * (size_t)g.items;
    k_face_div<T, TETRA><<<kFaceBlocks, 256, 0, s>>>(Pf, fi);
    blocks += kFaceBlocks;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (blocks_out) *blocks_out = blocks;
  return cudaSuccess;
}

template <typename T>
int residual_blocks(const ResParams<T>& P, int tetra) {
  (void)tetra;
  return fused_ok(P, false) ? fused_blocks(P) : RBLOCKS;
}

template <typename T, int TETRA, bool WITH_P, bool SYM>
static cudaError_t launch_res_t(const ResParams<T>& P, bool lo, cudaStream_t s, int* blocks_out) {
  const TileIdx tv = voxel_tiles(P.n);
  TileIdx tn;
  FaceIdx fi;
  interior_and_faces<T>(P, &tn, &fi);
  const bool inc = !WITH_P && P.inc;
  if (inc) {
    if (lo) k_stress_inc<T, TETRA, true, SYM><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
    else k_stress_inc<T, TETRA, false, SYM><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
  } else {
    if (P.slaw == 1) {
      if (lo) k_stress<T, TETRA, WITH_P, true, SYM, 1><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
      else k_stress<T, TETRA, WITH_P, false, SYM, 1><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
    } else if (P.slaw == 2) {
      if (lo) k_stress<T, TETRA, WITH_P, true, SYM, 2><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
      else k_stress<T, TETRA, WITH_P, false, SYM, 2><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
    } else if (P.slaw == 4) {
      if (lo) k_stress<T, TETRA, WITH_P, true, SYM, 4><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
      else k_stress<T, TETRA, WITH_P, false, SYM, 4><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
    } else {
      if (lo) k_stress<T, TETRA, WITH_P, true, SYM, 0><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
      else k_stress<T, TETRA, WITH_P, false, SYM, 0><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tv);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (inc) k_div<T, TETRA, false, SYM, true><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tn, fi);
  else k_div<T, TETRA, WITH_P, SYM, false><<<RBLOCKS, RTX * RTY, 0, s>>>(P, tn, fi);
  if (blocks_out) *blocks_out = RBLOCKS;
  return cudaGetLastError();
}

template <typename T, int TETRA>
static cudaError_t launch_res_s(const ResParams<T>& P, bool with_p, cudaStream_t s, int* b) {
  const bool lo = P.ulo[0] != nullptr;
  if (with_p) return P.sym ? launch_res_t<T, TETRA, true, true>(P, lo, s, b) : launch_res_t<T, TETRA, true, false>(P, lo, s, b);
  return P.sym ? launch_res_t<T, TETRA, false, true>(P, lo, s, b) : launch_res_t<T, TETRA, false, false>(P, lo, s, b);
}

template <typename T>
cudaError_t launch_residual(const ResParams<T>& P, int tetra, bool with_p, cudaStream_t s, int* blocks_out) {
  if (fused_ok(P, with_p))
    return tetra ? launch_fused_t<T, 1>(P, s, blocks_out) : launch_fused_t<T, 0>(P, s, blocks_out);
  return tetra ? launch_res_s<T, 1>(P, with_p, s, blocks_out) : launch_res_s<T, 0>(P, with_p, s, blocks_out);
}


template <typename T>
bool residual_one_pass(const ResParams<T>& P) {
  ResParams<T> Q = P;
  Q.two_pass = 0;
  return fused_ok(Q, false);
}

// ---- per-voxel evaluation shared by the output and statistics kernels ----
template <typename T, int TETRA, bool LO>
__device__ __forceinline__ int voxel_eval(const ResParams<T>& P, long long v, T Gt_out[2][9], T P_out[2][9],
                                          T (*stn)[10] = nullptr) {
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const int vx = (int)(v % n1);
  const long long r1 = v / n1;
  const int vy = (int)(r1 % n2);
  const int vz = (int)(r1 / n2);
  const int ph = P.phase[vx + vy * P.vy + (long long)vz * P.vz];
  const int law = __ldg(P.law_id + ph);
  const bool j2 = law == LAW_J2;
  const T* lc = P.law_c + (size_t)ph * LAWC;
  T uh[3][8], ul[3][8], nh[3][8], nl[3][8];
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    int gx = vx + (o & 1), gy = vy + ((o >> 1) & 1), gz = vz + (o >> 2);
    if (P.periodic[0] && gx == n1) gx = 0;
    if (P.periodic[1] && gy == n2) gy = 0;
    if (P.periodic[2] && gz == n3) gz = 0;
    const long long at = gx + gy * P.sy + (long long)gz * P.sz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uh[c][o] = P.u[c][at];
      ul[c][o] = LO ? P.ulo[c][at] : T(0);
      nh[c][o] = j2 ? P.un[c][at] : T(0);
      nl[c][o] = (j2 && LO) ? P.unlo[c][at] : T(0);
    }
  }
#pragma unroll
  for (int r = 0; r < (TETRA ? 2 : 1); ++r) {
    T Gf[9];
    law_grad<T, TETRA, LO>(P, false, uh, ul, r, vx, vy, vz, Gf, Gt_out[r]);  // total gradient (reported)
    if (j2) {
      T du[3][8], dl[3][8], Gd[9], Ginc[9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          du[c][o] = uh[c][o] - nh[c][o];
          dl[c][o] = ul[c][o] - nl[c][o];
        }
      law_grad<T, TETRA, LO>(P, true, du, dl, r, vx, vy, vz, Gd, Ginc);
      point_law<T>(P, law, lc, Ginc, r, v, (long long)n1 * n2 * n3, P_out[r], stn ? stn[r] : nullptr);
    } else {
      point_law<T>(P, law, lc, Gt_out[r], r, v, (long long)n1 * n2 * n3, P_out[r], stn ? stn[r] : nullptr);
    }
  }
  return law;
}

template <typename T, int TETRA, bool LO>
__global__ void k_commit(ResParams<T> P, T* __restrict__ out) {
  const long long nv = (long long)P.n[0] * P.n[1] * P.n[2];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    const int law = __ldg(P.law_id + P.phase[v]);
    if (law != LAW_J2 && law != LAW_CP && law != LAW_LOGJ2) continue;
    T Gt[2][9], Pp[2][9], stn[2][10];
    voxel_eval<T, TETRA, LO>(P, v, Gt, Pp, stn);
    const int nc = law == LAW_CP ? 10 : 7;
    for (int r = 0; r < (TETRA ? 2 : 1); ++r)
      for (int c = 0; c < nc; ++c) out[v + nv * (c + P.nst * r)] = stn[r][c];
  }
}

template <typename T>
cudaError_t launch_commit(const ResParams<T>& P, int tetra, T* out, cudaStream_t s) {
  if (!P.state) return cudaSuccess;
  const bool lo = P.ulo[0] != nullptr;
  if (tetra) {
    if (lo) k_commit<T, 1, true><<<1216, 256, 0, s>>>(P, out);
    else k_commit<T, 1, false><<<1216, 256, 0, s>>>(P, out);
  } else {
    if (lo) k_commit<T, 0, true><<<1216, 256, 0, s>>>(P, out);
    else k_commit<T, 0, false><<<1216, 256, 0, s>>>(P, out);
  }
  return cudaGetLastError();
}

template <typename T, int TETRA, bool LO>
__global__ void k_state_io(ResParams<T> P, T* __restrict__ out, const T* __restrict__ in) {
  const long long nv = (long long)P.n[0] * P.n[1] * P.n[2];
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    const int law = __ldg(P.law_id + P.phase[v]);
    if (law == LAW_CP) {  // stored as F^p - 1: read out F^p (row-major) and Gamma
      for (int r = 0; r < (TETRA ? 2 : 1); ++r) {
        T* st = P.state + v + nv * (P.nst * r);
        for (int c = 0; c < 9; ++c) {
          const T id = (c % 4 == 0) ? T(1) : T(0);
          if (out) out[v + nv * (c + P.nst * r)] = st[nv * c] + id;
          else st[nv * c] = in[v + nv * (c + P.nst * r)] - id;
        }
        if (out) out[v + nv * (9 + P.nst * r)] = st[nv * 9];
        else st[nv * 9] = in[v + nv * (9 + P.nst * r)];
      }
      continue;
    }
    if (law == LAW_LOGJ2) {  // stored as read out: H^p (6), p
      for (int r = 0; r < (TETRA ? 2 : 1); ++r) {
        T* st = P.state + v + nv * (P.nst * r);
        for (int c = 0; c < 7; ++c) {
          if (out) out[v + nv * (c + P.nst * r)] = st[nv * c];
          else st[nv * c] = in[v + nv * (c + P.nst * r)];
        }
      }
      continue;
    }
    if (law != LAW_J2) {
      if (out)
        for (int c = 0; c < P.nst * (TETRA ? 2 : 1); ++c) out[v + nv * c] = T(0);
      continue;
    }
    const int vx = (int)(v % n1);
    const long long r1 = v / n1;
    const int vy = (int)(r1 % n2), vz = (int)(r1 / n2);
    T uh[3][8], ul[3][8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      int gx = vx + (o & 1), gy = vy + ((o >> 1) & 1), gz = vz + (o >> 2);
      if (P.periodic[0] && gx == n1) gx = 0;
      if (P.periodic[1] && gy == n2) gy = 0;
      if (P.periodic[2] && gz == n3) gz = 0;
      const long long at = gx + gy * P.sy + (long long)gz * P.sz;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        uh[c][o] = P.u[c][at];
        ul[c][o] = LO ? P.ulo[c][at] : T(0);
      }
    }
#pragma unroll
    for (int r = 0; r < (TETRA ? 2 : 1); ++r) {
      T Gf[9], G[9];
      law_grad<T, TETRA, LO>(P, false, uh, ul, r, vx, vy, vz, Gf, G);
      const T es[6] = {G[0], G[4], G[8], T(0.5) * (G[5] + G[7]), T(0.5) * (G[2] + G[6]), T(0.5) * (G[1] + G[3])};
      T* st = P.state + v + nv * (P.nst * r);
      if (out) {
#pragma unroll
        for (int c = 0; c < 6; ++c) out[v + nv * (c + P.nst * r)] = es[c] - st[nv * c];
        out[v + nv * (6 + P.nst * r)] = st[nv * 6];
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) st[nv * c] = es[c] - in[v + nv * (c + P.nst * r)];
        st[nv * 6] = in[v + nv * (6 + P.nst * r)];
      }
    }
  }
}

template <typename T>
cudaError_t launch_state_io(const ResParams<T>& P, int tetra, T* out, const T* in, cudaStream_t s) {
  const bool lo = P.ulo[0] != nullptr;
  if (tetra) {
    if (lo) k_state_io<T, 1, true><<<1216, 256, 0, s>>>(P, out, in);
    else k_state_io<T, 1, false><<<1216, 256, 0, s>>>(P, out, in);
  } else {
    if (lo) k_state_io<T, 0, true><<<1216, 256, 0, s>>>(P, out, in);
    else k_state_io<T, 0, false><<<1216, 256, 0, s>>>(P, out, in);
  }
  return cudaGetLastError();
}

template <typename T, int TETRA, bool LO>
__global__ void k_voxel_fields(ResParams<T> P, T* __restrict__ gout, T* __restrict__ sout) {
  const long long nv = (long long)P.n[0] * P.n[1] * P.n[2];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    T Gt[2][9], Pp[2][9];
    voxel_eval<T, TETRA, LO>(P, v, Gt, Pp);
#pragma unroll
    for (int r = 0; r < (TETRA ? 2 : 1); ++r) {
      if (gout) {
#pragma unroll
        for (int i = 0; i < 9; ++i) gout[v + nv * (i + 9 * r)] = Gt[r][i];
      }
      if (sout && P.sym) {
        const int map[6] = {0, 4, 8, 5, 2, 1};  // 11, 22, 33, 23, 13, 12
#pragma unroll
        for (int c = 0; c < 6; ++c) sout[v + nv * (c + 6 * r)] = Pp[r][map[c]];
      } else if (sout) {
#pragma unroll
        for (int c = 0; c < 9; ++c) sout[v + nv * (c + 9 * r)] = Pp[r][c];
      }
    }
  }
}

template <typename T>
cudaError_t launch_voxel_fields(const ResParams<T>& P, int tetra, T* grad_out, T* stress_out, cudaStream_t s) {
  const bool lo = P.ulo[0] != nullptr;
  if (tetra) {
    if (lo) k_voxel_fields<T, 1, true><<<1216, 256, 0, s>>>(P, grad_out, stress_out);
    else k_voxel_fields<T, 1, false><<<1216, 256, 0, s>>>(P, grad_out, stress_out);
  } else {
    if (lo) k_voxel_fields<T, 0, true><<<1216, 256, 0, s>>>(P, grad_out, stress_out);
    else k_voxel_fields<T, 0, false><<<1216, 256, 0, s>>>(P, grad_out, stress_out);
  }
  return cudaGetLastError();
}

// ---- volume means of P and G (step report) ----
template <typename T, int TETRA, bool LO>
__global__ void __launch_bounds__(256) k_stats(ResParams<T> P, double* __restrict__ partial) {
  __shared__ double red[32];
  const long long nv = (long long)P.n[0] * P.n[1] * P.n[2];
  double acc[18];
#pragma unroll
  for (int i = 0; i < 18; ++i) acc[i] = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    T Gt[2][9], Pp[2][9];
    voxel_eval<T, TETRA, LO>(P, v, Gt, Pp);
#pragma unroll
    for (int r = 0; r < (TETRA ? 2 : 1); ++r)
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        acc[i] += (double)Pp[r][i];
        acc[9 + i] += (double)Gt[r][i];
      }
  }
  for (int i = 0; i < 18; ++i) {
    const double t = block_sum(acc[i], red);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * 18 + i] = t;
  }
}

template <typename T>
cudaError_t launch_stats(const ResParams<T>& P, int tetra, double* partial, int nblocks, cudaStream_t s) {
  const bool lo = P.ulo[0] != nullptr;
  if (tetra) {
    if (lo) k_stats<T, 1, true><<<nblocks, 256, 0, s>>>(P, partial);
    else k_stats<T, 1, false><<<nblocks, 256, 0, s>>>(P, partial);
  } else {
    if (lo) k_stats<T, 0, true><<<nblocks, 256, 0, s>>>(P, partial);
    else k_stats<T, 0, false><<<nblocks, 256, 0, s>>>(P, partial);
  }
  return cudaGetLastError();
}

}  // namespace fftm
