// Fixed-point residual: gradient -> constitutive law -> divergence, fused
// (Algorithm 1: grad u, P, D = div P + D*, the error; Eq. div_pol for p).
//
// A CTA owns a TX x TY tile of nodes in (x, y) and marches along z.  For each
// voxel plane it stages two node planes of u^f in shared memory, evaluates the
// gradient at the voxel points (HEX1: Eqs. D1HG-D3HG; TETRA2: Eqs.
// D1T1T2G-D3T1T2G) and the law, and keeps two voxel planes of P (and, for the
// test variant, tau = R0 : grad u^f - P with B0 = 2 mu0 G + lambda0 G (.) I,
// Sec. 2.6.3) in shared memory.  The divergence at a node plane (Remark 1:
// node m reads the voxels m + o - 1 with the same signs) yields D = div P, and
// the FP64 block partials of S_D = sum D^2 (transformed node components) and
// S_P = sum ||P||^2 / n_ppv.  The test variant also writes p = div tau.
//
// Stencil sums are formed as sums of differences of neighbouring values
// (u(o + e_i) - u(o) for HEX1; the paper's pairs for TETRA2), which are exact
// or nearly so in floating point for smooth fields, so the gradient carries
// the relative precision of the arithmetic instead of that of |u|.  In FP32
// the displacement is held as an unevaluated sum hi + lo of two floats (its
// low part carries what FP32 drops); both parts are differenced.
//
// TETRA2: tetrahedron T1 uses the four even-parity corners of the voxel, T2 the
// four odd-parity ones; along axis i the paper's two differences pair each
// corner c with o_i = 0 with c ^ (e_i + e_{i+1 mod 3}), over 2 h_i.  HEX1 pairs
// c with c + e_i over 4 h_i.  The residual D = 1/2 (div_T2 P^T1 + div_T1 P^T2)
// reads from the voxel at node offset o the T1 point for odd-parity o and the
// T2 point for even o, with weight sign / (4 h_i) -- the HEX1 weights.
//
// Ghost voxels (outside non-periodic faces) are never computed: a read is
// redirected to the mirror voxel inside, with the sign sigma(u_q, face) *
// (-1 if i is the face normal) on component (i, q), and with T1 <-> T2
// swapped once per face crossed (Sec. 2.2, Sec. 2.5.2).  Periodic axes wrap.
#include "fftm_internal.cuh"

namespace fftm {

enum { LAW_ISO = 0, LAW_CUBIC = 1, LAW_J2 = 2, LAW_B0 = 3 };

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

template <typename T, int TETRA, int TX, int TY, bool WITH_P, bool LO>
__global__ void __launch_bounds__(TX * TY) k_residual(ResParams<T> P) {
  constexpr int NPP = TETRA ? 2 : 1;
  constexpr int NE = WITH_P ? 18 : 9;  // P (9) [+ tau (9)] per voxel point
  constexpr int VX = TX + 1, VY = TY + 1, VPL = VX * VY;
  constexpr int NX = TX + 2, NY = TY + 2, NPL = NX * NY;
  constexpr int NLO = LO ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* nodes = reinterpret_cast<T*>(smem_raw);  // [NLO][2][3][NPL]
  T* vox = nodes + NLO * 2 * 3 * NPL;         // [2][NPP*NE][VPL]
  __shared__ double red[32];

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const int N1 = P.N[0], N2 = P.N[1], N3 = P.N[2];
  const int px = P.periodic[0], py = P.periodic[1], pz = P.periodic[2];
  const int zc0 = blockIdx.z * P.zchunk;
  const int zc1 = min(zc0 + P.zchunk, N3);
  double SD = 0.0, SP = 0.0;

  auto compute_plane = [&](int vz, int slot, bool owned) {
    // node planes vz and vz + 1 (wrapped on a periodic z)
    const int za = vz, zb = pz ? (vz + 1) % n3 : vz + 1;
    __syncthreads();
    for (int idx = tid; idx < NLO * 2 * 3 * NPL; idx += TX * TY) {
      const int e = idx % NPL;
      const int c = (idx / NPL) % 3;
      const int pl = (idx / (3 * NPL)) % 2;
      const int part = idx / (6 * NPL);
      int gx = x0 - 1 + e % NX, gy = y0 - 1 + e / NX;
      bool ok = true;
      if (px) gx = (gx + n1) % n1; else ok = ok && gx >= 0 && gx < N1;
      if (py) gy = (gy + n2) % n2; else ok = ok && gy >= 0 && gy < N2;
      const int gz = pl ? zb : za;
      const T* src = part ? P.ulo[c] : P.u[c];
      nodes[idx] = ok ? src[gx + gy * P.sy + (long long)gz * P.sz] : T(0);
    }
    __syncthreads();
    T* V = vox + slot * (NPP * NE * VPL);
    for (int e = tid; e < VPL; e += TX * TY) {
      const int lx = e % VX, ly = e / VX;
      const int vx = x0 - 1 + lx, vy = y0 - 1 + ly;
      if (vx >= n1 || vy >= n2) continue;
      if ((vx < 0 && !px) || (vy < 0 && !py)) continue;
      const int vxw = vx < 0 ? vx + n1 : vx, vyw = vy < 0 ? vy + n2 : vy;
      T uh[3][8], ul[3][8];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int at = (oz * 3 + c) * NPL + (ly + oy) * NX + lx + ox;
          uh[c][o] = nodes[at];
          ul[c][o] = LO ? nodes[6 * NPL + at] : T(0);
        }
      }
      const int ph = P.phase[vxw + vyw * P.vy + (long long)vz * P.vz];
      const int law = __ldg(P.law_id + ph);
      const T* lc = P.law_c + (size_t)ph * LAWC;
      const bool own = owned && lx >= 1 && ly >= 1;
#pragma unroll
      for (int r = 0; r < NPP; ++r) {
        T Gf[9], Gt[9], Pp[9];
        point_grad<T, TETRA, LO>(uh, ul, r, P.wgrad, Gf);
#pragma unroll
        for (int i = 0; i < 9; ++i) Gt[i] = Gf[i] + P.Gs[i];
        law_eval<T>(law, lc, Gt, Pp);
        T* dst = V + (r * NE) * VPL + e;
        double pn = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          dst[i * VPL] = Pp[i];
          pn += (double)Pp[i] * (double)Pp[i];
        }
        if (WITH_P) {
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              T t = P.two_mu0 * Gf[i * 3 + q] - Pp[i * 3 + q];
              if (i == q) t += P.lam0 * Gf[i * 3 + i];
              dst[(9 + i * 3 + q) * VPL] = t;
            }
        }
        if (own) SP += pn / NPP;
      }
    }
  };

  int prev = 0, cur = 1;
  if (zc0 >= 1) compute_plane(zc0 - 1, prev, false);
  else if (pz) compute_plane(n3 - 1, prev, false);

  for (int mz = zc0; mz < zc1; ++mz) {
    if (mz < n3) compute_plane(mz, cur, true);
    __syncthreads();
    const int lx = tid % TX, ly = tid / TX;
    const int mx = x0 + lx, my = y0 + ly;
    if (mx < N1 && my < N2) {
      // voxel read for corner offset o: pointer to its point values and the
      // ghost signs (ghost factor per (i, q) = sq[q] * (crossed axis i ? -1 : 1))
      const T* Vp[8];
      int crossm[8];
      T sqv[8][3];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
        const int vx = mx + ox - 1, vy = my + oy - 1, vz = mz + oz - 1;
        int tlx = lx + ox, tly = ly + oy;
        int slot = oz ? cur : prev;
        int cross = 0, sx = 0, sy = 0, sz = 0;
        if (!px) {
          if (vx < 0) { tlx += 1; cross |= 1; sx = 0; }
          else if (vx >= n1) { tlx -= 1; cross |= 1; sx = 1; }
        }
        if (!py) {
          if (vy < 0) { tly += 1; cross |= 2; sy = 0; }
          else if (vy >= n2) { tly -= 1; cross |= 2; sy = 1; }
        }
        if (!pz) {
          if (vz < 0) { slot = cur; cross |= 4; sz = 0; }
          else if (vz >= n3) { slot = prev; cross |= 4; sz = 1; }
        }
        int r = 0;
        if (TETRA) {
          r = ((ox + oy + oz) & 1) ? 0 : 1;  // odd corner -> T1 point (div_T2), even -> T2 (div_T1)
          if (__popc(cross) & 1) r ^= 1;
        }
        Vp[o] = vox + slot * (NPP * NE * VPL) + (r * NE) * VPL + tly * VX + tlx;
        crossm[o] = cross;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          int s = 1;
          if (cross & 1) s *= P.sgn[q][0][sx];
          if (cross & 2) s *= P.sgn[q][1][sy];
          if (cross & 4) s *= P.sgn[q][2][sz];
          sqv[o][q] = T(s);
        }
      }
      T Dq[3] = {T(0), T(0), T(0)}, pq[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          T s = T(0), st = T(0);
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            if ((o >> i) & 1) continue;
            const int o1 = o | (1 << i);
            const T f0 = ((crossm[o] >> i) & 1) ? -sqv[o][q] : sqv[o][q];
            const T f1 = ((crossm[o1] >> i) & 1) ? -sqv[o1][q] : sqv[o1][q];
            s += f1 * Vp[o1][(i * 3 + q) * VPL] - f0 * Vp[o][(i * 3 + q) * VPL];
            if (WITH_P) st += f1 * Vp[o1][(9 + i * 3 + q) * VPL] - f0 * Vp[o][(9 + i * 3 + q) * VPL];
          }
          Dq[q] += P.wdiv[i] * s;
          if (WITH_P) pq[q] += P.wdiv[i] * st;
        }
      }
      const long long off = mx + my * P.sy + (long long)mz * P.sz;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const bool dof = mx >= P.lo[q][0] && mx < P.hi[q][0] && my >= P.lo[q][1] && my < P.hi[q][1] &&
                         mz >= P.lo[q][2] && mz < P.hi[q][2];
        P.D[q][off] = dof ? Dq[q] : T(0);
        if (WITH_P) P.p[q][off] = dof ? pq[q] : T(0);
        if (dof) SD += (double)Dq[q] * (double)Dq[q];
      }
    }
    __syncthreads();
    const int t = prev;
    prev = cur;
    cur = t;
  }

  const double sd = block_sum(SD, red);
  const double sp = block_sum(SP, red);
  if (tid == 0) {
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    P.partial[2 * b] = sd;
    P.partial[2 * b + 1] = sp;
  }
}

template <typename T>
struct ResTile;
template <>
struct ResTile<float> { static constexpr int TX = 32, TY = 8; };
template <>
struct ResTile<double> { static constexpr int TX = 32, TY = 4; };

template <typename T>
static dim3 res_grid(const ResParams<T>& P, int* zchunk) {
  constexpr int TX = ResTile<T>::TX, TY = ResTile<T>::TY;
  const int bx = (P.N[0] + TX - 1) / TX, by = (P.N[1] + TY - 1) / TY;
  int chunks = (4 * 152 + bx * by - 1) / (bx * by);
  chunks = max(1, min(chunks, (P.N[2] + 7) / 8));
  const int zc = (P.N[2] + chunks - 1) / chunks;
  *zchunk = zc;
  return dim3(bx, by, (P.N[2] + zc - 1) / zc);
}

template <typename T>
int residual_blocks(const ResParams<T>& P, int tetra) {
  (void)tetra;
  int zc;
  dim3 g = res_grid<T>(P, &zc);
  return (int)(g.x * g.y * g.z);
}

template <typename T, int TETRA, bool WITH_P, bool LO>
static cudaError_t launch_res_t(ResParams<T> P, cudaStream_t s, int* blocks_out) {
  constexpr int TX = ResTile<T>::TX, TY = ResTile<T>::TY;
  constexpr int NPP = TETRA ? 2 : 1;
  constexpr int NE = WITH_P ? 18 : 9;
  int zc;
  dim3 grid = res_grid<T>(P, &zc);
  P.zchunk = zc;
  const size_t smem =
      sizeof(T) * ((LO ? 2 : 1) * 2 * 3 * (TX + 2) * (TY + 2) + 2 * NPP * NE * (TX + 1) * (TY + 1));
  auto kern = k_residual<T, TETRA, TX, TY, WITH_P, LO>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, TX * TY, smem, s>>>(P);
  if (blocks_out) *blocks_out = (int)(grid.x * grid.y * grid.z);
  return cudaGetLastError();
}

template <typename T, int TETRA>
static cudaError_t launch_res_s(const ResParams<T>& P, bool with_p, cudaStream_t s, int* b) {
  const bool lo = P.ulo[0] != nullptr;
  if (with_p) return lo ? launch_res_t<T, TETRA, true, true>(P, s, b) : launch_res_t<T, TETRA, true, false>(P, s, b);
  return lo ? launch_res_t<T, TETRA, false, true>(P, s, b) : launch_res_t<T, TETRA, false, false>(P, s, b);
}

template <typename T>
cudaError_t launch_residual(const ResParams<T>& P, int tetra, bool with_p, cudaStream_t s, int* blocks_out) {
  return tetra ? launch_res_s<T, 1>(P, with_p, s, blocks_out) : launch_res_s<T, 0>(P, with_p, s, blocks_out);
}

template cudaError_t launch_residual<float>(const ResParams<float>&, int, bool, cudaStream_t, int*);
template cudaError_t launch_residual<double>(const ResParams<double>&, int, bool, cudaStream_t, int*);
template int residual_blocks<float>(const ResParams<float>&, int);
template int residual_blocks<double>(const ResParams<double>&, int);

// ---- per-voxel evaluation shared by the output and statistics kernels ----
template <typename T, int TETRA, bool LO>
__device__ __forceinline__ void voxel_eval(const ResParams<T>& P, long long v, T Gt_out[2][9], T P_out[2][9]) {
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  const int vx = (int)(v % n1);
  const long long r1 = v / n1;
  const int vy = (int)(r1 % n2);
  const int vz = (int)(r1 / n2);
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
  const int ph = P.phase[vx + vy * P.vy + (long long)vz * P.vz];
  const int law = __ldg(P.law_id + ph);
  const T* lc = P.law_c + (size_t)ph * LAWC;
#pragma unroll
  for (int r = 0; r < (TETRA ? 2 : 1); ++r) {
    T Gf[9];
    point_grad<T, TETRA, LO>(uh, ul, r, P.wgrad, Gf);
#pragma unroll
    for (int i = 0; i < 9; ++i) Gt_out[r][i] = Gf[i] + P.Gs[i];
    law_eval<T>(law, lc, Gt_out[r], P_out[r]);
  }
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
      if (sout) {
        const int map[6] = {0, 4, 8, 5, 2, 1};  // 11, 22, 33, 23, 13, 12
#pragma unroll
        for (int c = 0; c < 6; ++c) sout[v + nv * (c + 6 * r)] = Pp[r][map[c]];
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
template cudaError_t launch_voxel_fields<float>(const ResParams<float>&, int, float*, float*, cudaStream_t);
template cudaError_t launch_voxel_fields<double>(const ResParams<double>&, int, double*, double*, cudaStream_t);

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
template cudaError_t launch_stats<float>(const ResParams<float>&, int, double*, int, cudaStream_t);
template cudaError_t launch_stats<double>(const ResParams<double>&, int, double*, int, cudaStream_t);

}  // namespace fftm
