// Axis passes of the 3D discrete transforms (Sec. 2.7.2: a 3D DT is three 1D
// DTs, x then y then z; the inverse runs z, y, x).
//
// One CTA transforms a tile of TP real pencils of one component along one
// axis (TP = 128 bytes of consecutive x for the y and z axes, TP consecutive
// rows for the x axis).  The tile goes through shared memory:
//
//   global --coalesced--> staging [j][pencil] --pre--> complex buffer
//   (digit-reversed) --in-place mixed-radix DIT FFT--> natural order
//   --post--> staging --coalesced--> global
//
// Two real pencils (a, b) share one complex pencil z = a + i b.  Each of the
// five Table 1 transforms and their inverses becomes one complex FFT of
// length M with O(M) pre/post-processing:
//   DFT    M = n : forward split of Z into the spectra of a and b, halfcomplex out
//   DCT-I  M = 2n: even extension, DFT is real                 (REDFT00)
//   DST-I  M = 2n: odd extension, DFT is imaginary              (RODFT00)
//   DCT-III M = 2n: Hermitian sequence x_j e^{+-i pi j/2n}, inverse DFT is real (REDFT01)
//   DST-III = (-1)^k DCT-III of the reversed input              (RODFT01)
//   DCT-II (inverse of DCT-III) = 2 Re(e^{-i pi k/2n} DFT_2n(x padded))  (REDFT10)
//   DST-II (inverse of DST-III) = DCT-II of (-1)^j x, reversed  (RODFT10)
// The fused z pass multiplies the z spectrum by the Green factor (Eqs.
// NSGO1_*, NSGO2_*) and runs the inverse z transform without leaving the SM.
#include "fftm_internal.cuh"

namespace fftm {

template <typename T>
using v2 = typename V2<T>::t;

template <typename T>
__device__ __forceinline__ v2<T> mk(T x, T y) {
  v2<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T>
__device__ __forceinline__ v2<T> cadd(v2<T> a, v2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ v2<T> csub(v2<T> a, v2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ v2<T> cmul(v2<T> a, v2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ v2<T> mul_mi(v2<T> a) { return mk<T>(a.y, -a.x); }  // a * (-i)

// R-point forward DFTs (kernel exp(-2 pi i rt / R)) in registers.
template <typename T>
__device__ __forceinline__ void dft2(v2<T>* x) {
  v2<T> a = x[0], b = x[1];
  x[0] = cadd<T>(a, b);
  x[1] = csub<T>(a, b);
}
template <typename T>
__device__ __forceinline__ void dft4(v2<T>& x0, v2<T>& x1, v2<T>& x2, v2<T>& x3) {
  v2<T> t0 = cadd<T>(x0, x2), t1 = csub<T>(x0, x2);
  v2<T> t2 = cadd<T>(x1, x3), t3 = mul_mi<T>(csub<T>(x1, x3));
  x0 = cadd<T>(t0, t2);
  x2 = csub<T>(t0, t2);
  x1 = cadd<T>(t1, t3);
  x3 = csub<T>(t1, t3);
}
template <typename T>
__device__ __forceinline__ void dft3(v2<T>* x) {
  const T h = T(0.86602540378443864676);  // sqrt(3)/2
  v2<T> t1 = cadd<T>(x[1], x[2]), t2 = csub<T>(x[1], x[2]);
  v2<T> m = mk<T>(x[0].x - T(0.5) * t1.x, x[0].y - T(0.5) * t1.y);
  v2<T> s = mk<T>(h * t2.y, -h * t2.x);  // -i sqrt(3)/2 (x1 - x2)
  x[0] = cadd<T>(x[0], t1);
  x[1] = cadd<T>(m, s);
  x[2] = csub<T>(m, s);
}
template <typename T>
__device__ __forceinline__ void dft8(v2<T>* x) {
  const T c = T(0.70710678118654752440);  // sqrt(1/2)
  v2<T> e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  v2<T> o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<T>(e0, e1, e2, e3);
  dft4<T>(o0, o1, o2, o3);
  o1 = mk<T>(c * (o1.x + o1.y), c * (o1.y - o1.x));   // * e^{-i pi/4}
  o2 = mul_mi<T>(o2);                                 // * e^{-i pi/2}
  o3 = mk<T>(c * (o3.y - o3.x), -c * (o3.x + o3.y));  // * e^{-3 i pi/4}
  x[0] = cadd<T>(e0, o0);
  x[4] = csub<T>(e0, o0);
  x[1] = cadd<T>(e1, o1);
  x[5] = csub<T>(e1, o1);
  x[2] = cadd<T>(e2, o2);
  x[6] = csub<T>(e2, o2);
  x[3] = cadd<T>(e3, o3);
  x[7] = csub<T>(e3, o3);
}

// In-place mixed-radix decimation-in-time FFT of PC complex pencils stored
// buf[m * PC + pc], input in digit-reversed order, output in natural order.
template <typename T, int PC>
__device__ void fft_stages(v2<T>* buf, const AxisPlan<T>& pl, const v2<T>* tw) {
  int Lp = 1;
  const int M = pl.M;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    const int Ls = Lp * R;
    const int nb = M / R;
    const int tstep = M / Ls;
    // b / Lp as a multiply-high: exact for b < 2^16 and 2 <= Lp <= 2^13 with
    // magic = ceil(2^32 / Lp) (the rounding excess b (magic Lp - 2^32) / 2^32 < 2^-16
    // stays below 1 / Lp); the first stage has Lp = 1
    const unsigned magic =
        Lp > 1 ? (unsigned)((0x100000000ull + (unsigned long long)Lp - 1) / (unsigned long long)Lp) : 0u;
    for (int idx = threadIdx.x; idx < nb * PC; idx += blockDim.x) {
      const int pc = idx % PC;
      const int b = idx / PC;
      const int g = Lp > 1 ? (int)__umulhi((unsigned)b, magic) : b;
      const int k = b - g * Lp;
      const int base = g * Ls + k;
      v2<T> x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < R) x[r] = buf[(base + r * Lp) * PC + pc];
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < 8; ++r)
          if (r < R) x[r] = cmul<T>(x[r], tw[r * k * tstep]);
      }
      if (R == 8) dft8<T>(x);
      else if (R == 4) dft4<T>(x[0], x[1], x[2], x[3]);
      else if (R == 3) dft3<T>(x);
      else dft2<T>(x);
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < R) buf[(base + r * Lp) * PC + pc] = x[r];
    }
    __syncthreads();
    Lp = Ls;
  }
}

// Complex work buffer: buf[m * PC + pc], pencils interleaved, FFT input digit-reversed.
template <int PC>
struct BufIx {
  static __device__ __forceinline__ int at(int pc, int m) { return m * PC + pc; }
};

// Staging accessors: stg[row * SP + pencil], row = position - lo.
template <typename T>
struct Stage {
  T* s;
  int SP;
  __device__ __forceinline__ T& at(int row, int p) const { return s[row * SP + p]; }
};

// Forward pre-processing: sequence value at index m for complex pencil pc.
template <typename T, int KIND>
__device__ __forceinline__ v2<T> pre_forward(const AxisPlan<T>& pl, const Stage<T>& st, int pc, int m,
                                             const v2<T>* qw) {
  const int n = pl.n;
  const int pa = 2 * pc, pb = pa + 1;
  switch (KIND) {
    case K_DFT:
      return mk<T>(st.at(m, pa), st.at(m, pb));
    case K_DCT1: {
      const int j = (m <= n) ? m : 2 * n - m;
      return mk<T>(st.at(j, pa), st.at(j, pb));
    }
    case K_DST1: {
      if (m == 0 || m == n) return mk<T>(T(0), T(0));
      if (m < n) return mk<T>(st.at(m - 1, pa), st.at(m - 1, pb));
      const int j = 2 * n - m;
      return mk<T>(-st.at(j - 1, pa), -st.at(j - 1, pb));
    }
    default: {  // DCT3 (rows j = 0..n-1) or DST3 (rows j-1 for nodes j = 1..n, read reversed)
      if (m == n) return mk<T>(T(0), T(0));
      const bool rev = (KIND == K_DST3);
      const int j = (m < n) ? m : 2 * n - m;  // index into the (reversed) input sequence
      const int row = rev ? (n - j) - 1 : j;  // DST3: x'_j = g_{n-j}, stored at row (n - j) - 1
      const v2<T> z = mk<T>(st.at(row, pa), st.at(row, pb));
      if (m == 0) return mk<T>(z.x, -z.y);  // conj(H_0)
      v2<T> w = qw[j];
      if (m > n) w.y = -w.y;
      const v2<T> h = cmul<T>(z, w);
      return mk<T>(h.x, -h.y);  // conj(H_m): the inverse DFT runs as conj(FFT(conj H))
    }
  }
}

// Forward post-processing: writes output row(s) of complex pencil pc for item k.
template <typename T, int KIND, int PC>
__device__ __forceinline__ void post_forward(const AxisPlan<T>& pl, const v2<T>* buf, const Stage<T>& st,
                                             int pc, int k) {
  using B = BufIx<PC>;
  const int n = pl.n;
  const int pa = 2 * pc, pb = pa + 1;
  switch (KIND) {
    case K_DFT: {  // k in [0, n/2]
      const v2<T> Zk = buf[B::at(pc, k)];
      const v2<T> Zn = buf[B::at(pc, (n - k) % n)];
      const T ax = T(0.5) * (Zk.x + Zn.x), ay = T(0.5) * (Zk.y - Zn.y);
      const T dx = Zk.x - Zn.x, dy = Zk.y + Zn.y;
      const T bx = T(0.5) * dy, by = T(-0.5) * dx;
      st.at(k, pa) = ax;
      st.at(k, pb) = bx;
      if (k > 0 && 2 * k < n) {
        st.at(n - k, pa) = ay;
        st.at(n - k, pb) = by;
      }
      break;
    }
    case K_DCT1: {  // k in [0, n]
      const v2<T> Y = buf[B::at(pc, k)];
      st.at(k, pa) = Y.x;
      st.at(k, pb) = Y.y;
      break;
    }
    case K_DST1: {  // k in [0, n-2], DFT bin k + 1
      const v2<T> Z = buf[B::at(pc, k + 1)];
      st.at(k, pa) = -Z.y;
      st.at(k, pb) = Z.x;
      break;
    }
    default: {  // DCT3 / DST3, k in [0, n-1]
      const v2<T> R = buf[B::at(pc, k)];
      const T sg = (KIND == K_DST3 && (k & 1)) ? T(-1) : T(1);
      st.at(k, pa) = sg * R.x;
      st.at(k, pb) = -sg * R.y;
      break;
    }
  }
}

// Inverse pre-processing: sequence value at index m for complex pencil pc.
template <typename T, int KIND>
__device__ __forceinline__ v2<T> pre_inverse(const AxisPlan<T>& pl, const Stage<T>& st, int pc, int m) {
  const int n = pl.n;
  const int pa = 2 * pc, pb = pa + 1;
  switch (KIND) {
    case K_DFT: {
      // halfcomplex rows -> spectra A (of a) and B (of b) at frequency m -> Z = A + i B
      T ax, ay, bx, by;
      if (m == 0 || 2 * m == n) {
        ax = st.at(m, pa); ay = T(0);
        bx = st.at(m, pb); by = T(0);
      } else if (2 * m < n) {
        ax = st.at(m, pa); ay = st.at(n - m, pa);
        bx = st.at(m, pb); by = st.at(n - m, pb);
      } else {
        ax = st.at(n - m, pa); ay = -st.at(m, pa);
        bx = st.at(n - m, pb); by = -st.at(m, pb);
      }
      const T zx = ax - by, zy = ay + bx;
      return mk<T>(zx, -zy);  // conj(Z): inverse DFT as conj(FFT(conj Z))
    }
    case K_DCT1:
    case K_DST1: {
      // DCT-I and DST-I are their own inverses up to 1/(2n)
      const int nn = n;
      if (KIND == K_DCT1) {
        const int j = (m <= nn) ? m : 2 * nn - m;
        return mk<T>(st.at(j, pa), st.at(j, pb));
      }
      if (m == 0 || m == nn) return mk<T>(T(0), T(0));
      if (m < nn) return mk<T>(st.at(m - 1, pa), st.at(m - 1, pb));
      const int j = 2 * nn - m;
      return mk<T>(-st.at(j - 1, pa), -st.at(j - 1, pb));
    }
    default: {  // DCT-II (inverse of DCT3) / DST-II via DCT-II of (-1)^m Y_m
      if (m >= n) return mk<T>(T(0), T(0));
      const T sg = (KIND == K_DST3 && (m & 1)) ? T(-1) : T(1);
      return mk<T>(sg * st.at(m, pa), sg * st.at(m, pb));
    }
  }
}

// Inverse post-processing: output item j of complex pencil pc.
template <typename T, int KIND, int PC>
__device__ __forceinline__ void post_inverse(const AxisPlan<T>& pl, const v2<T>* buf, const Stage<T>& st,
                                             int pc, int j, const v2<T>* qw) {
  using B = BufIx<PC>;
  const int n = pl.n;
  const int pa = 2 * pc, pb = pa + 1;
  switch (KIND) {
    case K_DFT: {  // j in [0, n)
      const v2<T> R = buf[B::at(pc, j)];
      st.at(j, pa) = R.x;
      st.at(j, pb) = -R.y;
      break;
    }
    case K_DCT1: {  // j in [0, n]
      const v2<T> Y = buf[B::at(pc, j)];
      st.at(j, pa) = Y.x;
      st.at(j, pb) = Y.y;
      break;
    }
    case K_DST1: {  // output rows j in [0, n-2] <- bin j + 1
      const v2<T> Z = buf[B::at(pc, j + 1)];
      st.at(j, pa) = -Z.y;
      st.at(j, pb) = Z.x;
      break;
    }
    default: {  // DCT-II item j in [0, n)
      const v2<T> Zj = buf[B::at(pc, j)];
      const v2<T> Zc = buf[B::at(pc, (2 * n - j) % (2 * n))];
      const T ax = T(0.5) * (Zj.x + Zc.x), ay = T(0.5) * (Zj.y - Zc.y);
      const T dx = Zj.x - Zc.x, dy = Zj.y + Zc.y;
      const T bx = T(0.5) * dy, by = T(-0.5) * dx;
      const v2<T> w = qw[j];  // (cos, sin)(pi j / 2n)
      const T oa = T(2) * (ax * w.x + ay * w.y);
      const T ob = T(2) * (bx * w.x + by * w.y);
      const int row = (KIND == K_DST3) ? (n - j) - 1 : j;  // DST-II: node n - j, row n - j - 1
      st.at(row, pa) = oa;
      st.at(row, pb) = ob;
      break;
    }
  }
}

// The pre- and post-processing loops of one CTA with the transform kind resolved
// at compile time (one switch per CTA instead of one per element).
template <typename T, int PC, int KIND>
__device__ __forceinline__ void pre_loop(const AxisPlan<T>& pl, const Stage<T>& st, v2<T>* buf, const int16_t* perm,
                                         const v2<T>* qw, bool inverse) {
  using B = BufIx<PC>;
  const int M = pl.M;
  if (inverse) {
    for (int idx = threadIdx.x; idx < M * PC; idx += blockDim.x) {
      const int pc = idx % PC, m = idx / PC;
      buf[B::at(pc, perm[m])] = pre_inverse<T, KIND>(pl, st, pc, m);
    }
  } else {
    for (int idx = threadIdx.x; idx < M * PC; idx += blockDim.x) {
      const int pc = idx % PC, m = idx / PC;
      buf[B::at(pc, perm[m])] = pre_forward<T, KIND>(pl, st, pc, m, qw);
    }
  }
}

template <typename T, int PC, int KIND>
__device__ __forceinline__ void post_loop(const AxisPlan<T>& pl, const Stage<T>& st, const v2<T>* buf,
                                          const v2<T>* qw, bool inverse) {
  if (inverse) {
    for (int idx = threadIdx.x; idx < pl.L * PC; idx += blockDim.x) {
      const int pc = idx % PC, j = idx / PC;
      post_inverse<T, KIND, PC>(pl, buf, st, pc, j, qw);
    }
  } else {
    const int nitems = KIND == K_DFT ? pl.n / 2 + 1 : pl.L;
    for (int idx = threadIdx.x; idx < nitems * PC; idx += blockDim.x) {
      const int pc = idx % PC, k = idx / PC;
      post_forward<T, KIND, PC>(pl, buf, st, pc, k);
    }
  }
}

template <typename T, int PC>
__device__ __forceinline__ void pre_dispatch(const AxisPlan<T>& pl, const Stage<T>& st, v2<T>* buf,
                                             const int16_t* perm, const v2<T>* qw, bool inverse) {
  switch (pl.kind) {
    case K_DFT: pre_loop<T, PC, K_DFT>(pl, st, buf, perm, qw, inverse); break;
    case K_DCT1: pre_loop<T, PC, K_DCT1>(pl, st, buf, perm, qw, inverse); break;
    case K_DST1: pre_loop<T, PC, K_DST1>(pl, st, buf, perm, qw, inverse); break;
    case K_DCT3: pre_loop<T, PC, K_DCT3>(pl, st, buf, perm, qw, inverse); break;
    default: pre_loop<T, PC, K_DST3>(pl, st, buf, perm, qw, inverse); break;
  }
}

template <typename T, int PC>
__device__ __forceinline__ void post_dispatch(const AxisPlan<T>& pl, const Stage<T>& st, const v2<T>* buf,
                                              const v2<T>* qw, bool inverse) {
  switch (pl.kind) {
    case K_DFT: post_loop<T, PC, K_DFT>(pl, st, buf, qw, inverse); break;
    case K_DCT1: post_loop<T, PC, K_DCT1>(pl, st, buf, qw, inverse); break;
    case K_DST1: post_loop<T, PC, K_DST1>(pl, st, buf, qw, inverse); break;
    case K_DCT3: post_loop<T, PC, K_DCT3>(pl, st, buf, qw, inverse); break;
    default: post_loop<T, PC, K_DST3>(pl, st, buf, qw, inverse); break;
  }
}

template <typename T>
__device__ __forceinline__ T green_factor(const PassParams<T>& P, int q, int kx, int ky, int kz) {
  const T sx = P.S2[q][0][kx], cx = P.C2[q][0][kx];
  const T sy = P.S2[q][1][ky], cy = P.C2[q][1][ky];
  const T sz = P.S2[q][2][kz], cz = P.C2[q][2][kz];
  T a0 = P.hf[0] * sx * cy * cz;
  T a1 = P.hf[1] * cx * sy * cz;
  T a2 = P.hf[2] * cx * cy * sz;
  if (P.tetra) {
    a0 += P.hf[0] * cx * sy * sz;
    a1 += P.hf[1] * sx * cy * sz;
    a2 += P.hf[2] * sx * sy * cz;
  }
  const T aq = (q == 0) ? a0 : ((q == 1) ? a1 : a2);
  const T den = P.two_mu0 * (a0 + a1 + a2) + P.lam0 * aq;
  return den > T(0) ? -P.gscale[q] / den : T(0);
}

// Tile geometry: TP real pencils per CTA (128 bytes of T).
template <typename T>
struct TileCfg {
  static constexpr int TP = 128 / sizeof(T);
  static constexpr int PC = TP / 2;
  static constexpr int SP = TP + 1;
};

constexpr int PASS_THREADS = 512;

template <typename T, int AXIS, int FUSED>
__global__ void __launch_bounds__(PASS_THREADS) k_pass(PassParams<T> P) {
  if (P.stop && *P.stop) return;
  constexpr int TP = TileCfg<T>::TP;
  constexpr int PC = TileCfg<T>::PC;
  constexpr int SP = TileCfg<T>::SP;
  const int q = blockIdx.y;
  const AxisPlan<T>& pl = P.plan[q];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = pl.M;
  v2<T>* buf = reinterpret_cast<v2<T>*>(smem_raw);
  v2<T>* tw = buf + (size_t)M * PC;
  v2<T>* qw = tw + M;
  int16_t* perm = reinterpret_cast<int16_t*>(qw + (pl.n + 1));
  T* stg_raw = reinterpret_cast<T*>(smem_raw) + 0;  // placed after perm, aligned below
  {
    size_t off = (size_t)M * PC * sizeof(v2<T>) + (size_t)M * sizeof(v2<T>) + (size_t)(pl.n + 1) * sizeof(v2<T>) +
                 (size_t)M * sizeof(int16_t);
    off = (off + 15) & ~(size_t)15;
    stg_raw = reinterpret_cast<T*>(smem_raw + off);
  }
  Stage<T> st{stg_raw, SP};

  // ---- tile geometry ----
  const int N1 = P.N[0], N2 = P.N[1], N3 = P.N[2];
  const long long sx = P.stride[0], sy = P.stride[1], sz = P.stride[2];
  long long base0 = 0;
  long long pstride = 0;  // distance between consecutive pencils (axes 1, 2)
  long long estride = 0;  // distance between consecutive elements of a pencil
  int npen = TP;
  int row0 = 0;
  int x0 = 0, yfix = 0;
  if (AXIS == 0) {
    row0 = blockIdx.x * TP;
    npen = min(TP, N2 * N3 - row0);
    estride = sx;
  } else {
    const int ntx = (N1 + TP - 1) / TP;
    x0 = (blockIdx.x % ntx) * TP;
    const int other = blockIdx.x / ntx;
    npen = min(TP, N1 - x0);
    pstride = sx;
    if (AXIS == 1) {
      base0 = x0 * sx + (long long)other * sz;
      estride = sy;
    } else {
      yfix = other;
      base0 = x0 * sx + (long long)other * sy;
      estride = sz;
    }
  }
  if (FUSED) {
    // a y position outside the component's y range holds zeros and stays zero
    const int ky = yfix - P.flo[q][1];
    if (ky < 0 || ky >= P.fL[q][1]) return;
  }

  // ---- tables ----
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    cp_async_elem<T>(&tw[i].x, &pl.tw[i].x);
    cp_async_elem<T>(&tw[i].y, &pl.tw[i].y);
    perm[i] = pl.perm[i];
  }
  for (int i = threadIdx.x; i <= pl.n; i += blockDim.x) {
    cp_async_elem<T>(&qw[i].x, &pl.qw[i].x);
    cp_async_elem<T>(&qw[i].y, &pl.qw[i].y);
  }

  const T* __restrict__ in = P.in[q];
  T* __restrict__ out = P.out[q];
  const int L = pl.L, lo = pl.lo;

  // ---- load: global -> staging (asynchronous copies, all in flight at once) ----
  if (AXIS == 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int p = warp; p < TP; p += PASS_THREADS / 32) {
      if (p < npen) {
        const int r = row0 + p;
        const int y = r % N2, z = r / N2;
        const T* src = in + (long long)y * sy + (long long)z * sz + (long long)lo * estride;
        for (int j = lane; j < L; j += 32) cp_async_elem<T>(&st.at(j, p), src + (long long)j * estride);
      } else {
        for (int j = lane; j < L; j += 32) st.at(j, p) = T(0);
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < L * TP; idx += blockDim.x) {
      const int p = idx % TP;
      const int j = idx / TP;
      if (p < npen) cp_async_elem<T>(&st.at(j, p), in + base0 + p * pstride + (long long)(lo + j) * estride);
      else st.at(j, p) = T(0);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  const bool inv_first = (P.inverse != 0) && !FUSED;
  // ---- forward (or the inverse when not fused) ----
  pre_dispatch<T, PC>(pl, st, buf, perm, qw, inv_first);
  __syncthreads();
  fft_stages<T, PC>(buf, pl, tw);
  post_dispatch<T, PC>(pl, st, buf, qw, inv_first);
  __syncthreads();

  if (FUSED) {
    // ---- Green factor on the (kx, ky, kz) spectrum, then inverse z ----
    const int ky = yfix - P.flo[q][1];
    for (int idx = threadIdx.x; idx < L * TP; idx += blockDim.x) {
      const int p = idx % TP;
      const int kz = idx / TP;
      const int kx = x0 + p - P.flo[q][0];
      T g = T(0);
      if (p < npen && kx >= 0 && kx < P.fL[q][0]) g = green_factor<T>(P, q, kx, ky, kz);
      st.at(kz, p) *= g;
    }
    __syncthreads();
    pre_dispatch<T, PC>(pl, st, buf, perm, qw, true);
    __syncthreads();
    fft_stages<T, PC>(buf, pl, tw);
    post_dispatch<T, PC>(pl, st, buf, qw, true);
    __syncthreads();
  }

  // ---- store: staging -> global ----
  const T sc = P.scale[q];
  if (AXIS == 0) {
    const T* __restrict__ bh = P.base[q];
    const T* __restrict__ bl = P.base_lo[q];
    T* __restrict__ ol = P.out_lo[q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int p = warp; p < npen; p += PASS_THREADS / 32) {
      const int r = row0 + p;
      const int y = r % N2, z = r / N2;
      const long long at0 = (long long)y * sy + (long long)z * sz + (long long)lo * estride;
      for (int j = lane; j < L; j += 32) {
        const long long at = at0 + (long long)j * estride;
        const T v = sc * st.at(j, p);
        if (bh == nullptr) {
          out[at] = v;
        } else if (ol == nullptr) {
          out[at] = bh[at] + v;
        } else {
          // (hi, lo) = (bh, bl) + v: error-free sum of the high parts (TwoSum), low parts
          // gathered, then renormalised so that |lo| stays below half an ulp of hi
          const T a = bh[at];
          const T s1 = a + v;
          const T bb = s1 - a;
          const T e = (a - (s1 - bb)) + (v - bb);
          const T t = bl[at] + e;
          const T h = s1 + t;
          out[at] = h;
          ol[at] = t - (h - s1);
        }
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < L * TP; idx += blockDim.x) {
      const int p = idx % TP;
      const int j = idx / TP;
      if (p < npen) out[base0 + p * pstride + (long long)(lo + j) * estride] = sc * st.at(j, p);
    }
  }
}

template <typename T>
static size_t pass_smem(int maxM, int maxL, int maxn) {
  constexpr int PC = TileCfg<T>::PC;
  constexpr int SP = TileCfg<T>::SP;
  size_t off = (size_t)maxM * PC * sizeof(v2<T>) + (size_t)maxM * sizeof(v2<T>) + (size_t)(maxn + 1) * sizeof(v2<T>) +
               (size_t)maxM * sizeof(int16_t);
  off = (off + 15) & ~(size_t)15;
  return off + (size_t)maxL * SP * sizeof(T);
}

template <typename T, int AXIS, int FUSED>
static cudaError_t launch_one(const PassParams<T>& P, size_t smem, cudaStream_t s) {
  constexpr int TP = TileCfg<T>::TP;
  auto kern = k_pass<T, AXIS, FUSED>;
  // the same opt-in limit for every problem: the attribute is per function, so a
  // per-problem value could be lowered by another thread between its set and our launch
  (void)smem;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if (AXIS == 0) grid.x = (unsigned)((P.N[1] * P.N[2] + TP - 1) / TP);
  else grid.x = (unsigned)(((P.N[0] + TP - 1) / TP) * (AXIS == 1 ? P.N[2] : P.N[1]));
  grid.y = 3;
  kern<<<grid, PASS_THREADS, smem, s>>>(P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass(const PassParams<T>& P, int maxM, int maxL, int maxn, cudaStream_t s) {
  const size_t smem = pass_smem<T>(maxM, maxL, maxn);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (P.fused) {
    if (P.axis != 2) return cudaErrorInvalidValue;
    return launch_one<T, 2, 1>(P, smem, s);
  }
  if (P.axis == 0) return launch_one<T, 0, 0>(P, smem, s);
  if (P.axis == 1) return launch_one<T, 1, 0>(P, smem, s);
  return launch_one<T, 2, 0>(P, smem, s);
}

template cudaError_t launch_pass<float>(const PassParams<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_pass<double>(const PassParams<double>&, int, int, int, cudaStream_t);

// ---- standalone Green factor on a spectral field ----
template <typename T>
__global__ void k_green(GreenParams<T> P) {
  const int q = blockIdx.y;
  const long long total = (long long)P.N[0] * P.N[1] * P.N[2];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % P.N[0]);
    const long long r = i / P.N[0];
    const int y = (int)(r % P.N[1]);
    const int z = (int)(r / P.N[1]);
    const int kx = x - P.flo[q][0], ky = y - P.flo[q][1], kz = z - P.flo[q][2];
    const long long off = x + y * P.sy + z * P.sz;
    if (kx < 0 || ky < 0 || kz < 0 || kx >= P.fL[q][0] || ky >= P.fL[q][1] || kz >= P.fL[q][2]) {
      P.f[q][off] = T(0);
      continue;
    }
    const T sx = P.S2[q][0][kx], cx = P.C2[q][0][kx];
    const T sy = P.S2[q][1][ky], cy = P.C2[q][1][ky];
    const T sz = P.S2[q][2][kz], cz = P.C2[q][2][kz];
    T a0 = P.hf[0] * sx * cy * cz, a1 = P.hf[1] * cx * sy * cz, a2 = P.hf[2] * cx * cy * sz;
    if (P.tetra) {
      a0 += P.hf[0] * cx * sy * sz;
      a1 += P.hf[1] * sx * cy * sz;
      a2 += P.hf[2] * sx * sy * cz;
    }
    const T aq = (q == 0) ? a0 : ((q == 1) ? a1 : a2);
    const T den = P.two_mu0 * (a0 + a1 + a2) + P.lam0 * aq;
    P.f[q][off] *= (den > T(0) ? -P.gscale[q] / den : T(0));
  }
}

template <typename T>
cudaError_t launch_green(const GreenParams<T>& P, cudaStream_t s) {
  dim3 grid(1216, 3);
  k_green<T><<<grid, 256, 0, s>>>(P);
  return cudaGetLastError();
}
template cudaError_t launch_green<float>(const GreenParams<float>&, cudaStream_t);
template cudaError_t launch_green<double>(const GreenParams<double>&, cudaStream_t);

}  // namespace fftm
