// The C0 discrete Green operator (Sec. 2.6.1): reference stiffness C0 : grad u = 2 mu0 grad u
// + lambda0 tr(grad u) 1 (Eq. TF_C0_behavior).  With HEX1 its symbol on the real DCT-I / DST-I
// coefficients of normal-mixed BCs (Eq. SGO_BCs) is -(2 mu0 |xi|^2 I + lambda0 v (x) v), with
// (xi_H)_a = (2/h_a) sin(xi_a/2) prod_{b != a} cos(xi_b/2) (Eq. modified_freq_hex1) and
// v_q = tau_q (xi_H)_q, tau_q = -1 for a component symmetric about the faces normal to q and +1
// for an anti-symmetric one (the sign a derivative along q gives between the cosine and sine
// series).  Its inverse is the rank-one correction of Eq. FourierSGO_HEX1:
//     u_hat = -(p_hat - lambda0 / (2 mu0 + lambda0) (v . p_hat) v / |xi|^2) / (2 mu0 |xi|^2),
// zero where |xi|^2 vanishes.  TETRA2 (Eqs. p_u_tetra2, FourierSGO_TETRA2_1/2): with
// xi_T2 = xi_H + i xi' the coupling is lambda0 [(u . v) v + (u . w) w], w_q = tau_q xi'_q,
// (xi')_a = (2/h_a) cos(xi_a/2) prod_{b != a} sin(xi_b/2), and |xi|^2 = |xi_H|^2 + |xi'|^2; the
// rank-two correction is inverted through its 2 x 2 system (the paper's p_int pair, written on
// real vectors):  u = -(p - lambda0 [y1 v + y2 w]) / (2 mu0 |xi|^2) with
// (2 mu0 |xi|^2 I + lambda0 [v w]^T [v w]) y = [v . p, w . p].  The coefficients of the three
// components sit at the same node position for the same frequency (DCT-I and DST-I alike,
// xi = pi m / n), so one thread takes one node position and all three components; positions
// outside a component's range hold no coefficient of it (0 in, 0 out).
#include "fftm_internal.cuh"

namespace fftm {

template <typename T>
__global__ void __launch_bounds__(256) k_green_c0(const C0Params<T> P) {
  if (P.stop && *P.stop) return;
  const long long tot = (long long)P.N[0] * P.N[1] * P.N[2];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % P.N[0]);
    const long long r = i / P.N[0];
    const int y = (int)(r % P.N[1]), z = (int)(r / P.N[1]);
    const long long off = x + y * P.sy + z * P.sz;
    const T sx = P.s[0][x], cx = P.c[0][x];
    const T sy = P.s[1][y], cy = P.c[1][y];
    const T sz = P.s[2][z], cz = P.c[2][z];
    const T xi[3] = {P.hf[0] * sx * cy * cz, P.hf[1] * cx * sy * cz, P.hf[2] * cx * cy * sz};
    const T xp[3] = {P.hf[0] * cx * sy * sz, P.hf[1] * sx * cy * sz, P.hf[2] * sx * sy * cz};
    T xx = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    if (P.tetra) xx += xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2];
    bool in[3];
    T pv[3], v[3], w[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      in[q] = x >= P.lo[q][0] && x < P.hi[q][0] && y >= P.lo[q][1] && y < P.hi[q][1] && z >= P.lo[q][2] &&
              z < P.hi[q][2];
      pv[q] = in[q] ? P.f[q][off] : T(0);
      v[q] = P.tau[q] * xi[q];
      w[q] = P.tetra ? P.tau[q] * xp[q] : T(0);
    }
    const T vp = v[0] * pv[0] + v[1] * pv[1] + v[2] * pv[2];
    if (!P.tetra) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (!in[q]) continue;
        P.f[q][off] = xx > T(0) ? -P.gscale[q] * (pv[q] - P.beta * vp * v[q] / xx) / (P.two_mu0 * xx) : T(0);
      }
    } else {
      const T wp = w[0] * pv[0] + w[1] * pv[1] + w[2] * pv[2];
      const T vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      const T ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
      const T vw = v[0] * w[0] + v[1] * w[1] + v[2] * w[2];
      const T al = P.two_mu0 * xx, k11 = al + P.lam0 * vv, k22 = al + P.lam0 * ww, k12 = P.lam0 * vw;
      const T det = k11 * k22 - k12 * k12;
      const T y1 = det > T(0) ? (k22 * vp - k12 * wp) / det : T(0);
      const T y2 = det > T(0) ? (k11 * wp - k12 * vp) / det : T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (!in[q]) continue;
        P.f[q][off] = xx > T(0) ? -P.gscale[q] * (pv[q] - P.lam0 * (y1 * v[q] + y2 * w[q])) / al : T(0);
      }
    }
  }
}

template <typename T>
cudaError_t launch_green_c0(const C0Params<T>& P, cudaStream_t s) {
  k_green_c0<T><<<1216, 256, 0, s>>>(P);
  return cudaGetLastError();
}
template cudaError_t launch_green_c0<float>(const C0Params<float>&, cudaStream_t);
template cudaError_t launch_green_c0<double>(const C0Params<double>&, cudaStream_t);

}  // namespace fftm
