// Reductions, Anderson acceleration on p, and field (un)packing.
//
// Anderson acceleration on p (Sec. 2.3, Algorithm 1).  With couples (q_j, g_j),
// g_j = p_{j+1} the polarisation divergence produced by the transformed field
// q_j, the residual of a couple is f_j = g_j - q_j and the accelerated field
// is sum_j c_j g_j with c = argmin || sum_j c_j f_j ||_2, sum_j c_j = 1.  Since
// the Green operator inverts div(R0 : grad .) exactly on the transformed
// fields, q_j = div(R0 : grad u^{j+1}) and f_j = -D^{j+1}: the same step reads
// u_new = sum_k c_k u^k - Gamma(sum_k c_k D^k) with c = argmin ||sum_k c_k D^k||
// over the last iterates u^k and their residuals D^k.  That is the form used
// here (it keeps the rounding of the update relative to the residual).  The
// normal equations of the differences D_k - D_last are accumulated in FP64
// and solved by Cholesky in FP64 by one thread; a pivot below `pivot_tol`
// times its diagonal entry rejects the step (c = e_last).
#include <math_constants.h>

#include "fftm_internal.cuh"

namespace fftm {

// Sum `nvals` doubles over `nblocks` rows (fixed order: deterministic).
__global__ void k_reduce(const double* __restrict__ partial, int nblocks, int nvals, double* __restrict__ out,
                         const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double red[256];
  for (int v = 0; v < nvals; ++v) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * nvals + v];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = red[0];
    __syncthreads();
  }
}

cudaError_t launch_reduce_norms(const double* partial, int nblocks, int nvals, double* out, cudaStream_t s,
                                const int* stop) {
  k_reduce<<<1, 256, 0, s>>>(partial, nblocks, nvals, out, stop);
  return cudaGetLastError();
}

// The convergence test of Algorithm 1 on the device: err = h1 sqrt(S_D / S_P) (Eq.
// equilibrium_condition; +inf while S_P is 0 under a non-zero S_D, which only means "not yet"),
// recorded at err_hist[m]; the step stops when err < tol (1), on a non-finite norm (2) or at the
// iteration limit (3), else the next iteration is m + 1.
__global__ void k_check(const double* __restrict__ sums, int* __restrict__ ctl, double* __restrict__ err_hist,
                        double tol, int max_iter, double h1) {
  if (ctl[0]) return;
  const int m = ctl[1];
  const double sd = sums[0], sp = sums[1];
  const double err = sp > 0.0 ? h1 * sqrt(sd / sp) : (sd == 0.0 ? 0.0 : CUDART_INF);
  err_hist[m] = err;
  ctl[2] = m;
  if (isnan(err) || isinf(sd) || isinf(sp) || isnan(sd) || isnan(sp)) ctl[0] = 2;
  else if (err < tol) ctl[0] = 1;
  else if (m >= max_iter) ctl[0] = 3;
  else ctl[1] = m + 1;
}

cudaError_t launch_check(const double* sums, int* ctl, double* err_hist, double tol, int max_iter, double h1,
                         cudaStream_t s) {
  k_check<<<1, 1, 0, s>>>(sums, ctl, err_hist, tol, max_iter, h1);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_copy(T* d0, T* d1, T* d2, const T* s0, const T* s1, const T* s2, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    d0[i] = s0[i];
    d1[i] = s1[i];
    d2[i] = s2[i];
  }
}

template <typename T>
cudaError_t launch_copy_fields(T* const dst[3], const T* const src[3], long long count, cudaStream_t s) {
  k_copy<T><<<152 * 8, 256, 0, s>>>(dst[0], dst[1], dst[2], src[0], src[1], src[2], count);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_axpy(T* d0, T* d1, T* d2, const T* a0, const T* a1, const T* a2, const T* b0, const T* b1,
                       const T* b2, T alpha, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    d0[i] = a0[i] + alpha * b0[i];
    d1[i] = a1[i] + alpha * b1[i];
    d2[i] = a2[i] + alpha * b2[i];
  }
}

template <typename T>
cudaError_t launch_axpy_fields(T* const dst[3], const T* const a[3], const T* const b[3], T alpha, long long count,
                               cudaStream_t s) {
  k_axpy<T><<<152 * 8, 256, 0, s>>>(dst[0], dst[1], dst[2], a[0], a[1], a[2], b[0], b[1], b[2], alpha, count);
  return cudaGetLastError();
}

int gram_blocks(long long count) {
  (void)count;
  return 152 * 4;
}

// Normal matrix of the residual differences d_k = D_k - D_last (k < last) and
// the right-hand side <d_k, D_last>, formed from explicit differences (no
// Gram-entry cancellation) and reduced in FP64 across threads and blocks.
template <typename T>
struct GramArgs {
  const T* D[4][3];
};

// Accumulator of a sum of products: FP64 for double data; for float data an
// unevaluated pair (hi, lo) of floats updated with error-free transformations
// (TwoProduct through fma, TwoSum), which keeps about twice FP32's precision
// without the FP64 pipe (whose rate is a small fraction of FP32's on this GPU).
template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s += (double)a * (double)b; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);  // exact error of the product
    const float s = hi + p;
    const float bb = s - hi;
    const float se = (hi - (s - bb)) + (p - bb);  // exact error of the sum
    hi = s;
    lo += se + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
__global__ void __launch_bounds__(256) k_gram(GramArgs<T> A, int m, long long count, double* __restrict__ partial,
                                              const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double red[8][9];
  DotAcc<T> acc[9];
  const int L = m - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T v[4], d[3];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = (j < m) ? A.D[j][c][i] : T(0);
      T last = v[0];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j == L) last = v[j];
#pragma unroll
      for (int j = 0; j < 3; ++j) d[j] = (j < L) ? v[j] - last : T(0);
      acc[0].add(d[0], d[0]);
      acc[1].add(d[0], d[1]);
      acc[2].add(d[0], d[2]);
      acc[3].add(d[1], d[1]);
      acc[4].add(d[1], d[2]);
      acc[5].add(d[2], d[2]);
      acc[6].add(d[0], last);
      acc[7].add(d[1], last);
      acc[8].add(d[2], last);
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double v = acc[k].value();
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (l == 0) red[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
    partial[(size_t)blockIdx.x * 9 + threadIdx.x] = t;
  }
}

template <typename T>
cudaError_t launch_gram(const T* const D[4][3], int m, long long count, double* partial, int nblocks,
                        cudaStream_t s, const int* stop) {
  GramArgs<T> A;
  for (int j = 0; j < 4; ++j)
    for (int c = 0; c < 3; ++c) A.D[j][c] = (j < m) ? D[j][c] : D[0][c];
  k_gram<T><<<nblocks, 256, 0, s>>>(A, m, count, partial, stop);
  return cudaGetLastError();
}

// Reduce the partials; solve (d^T d) gamma = -(d^T D_last) by Cholesky in FP64;
// c_k = gamma_k (k < last), c_last = 1 - sum gamma.  A pivot below pivot_tol
// times its diagonal entry rejects the step: c = e_last.
__global__ void k_anderson_solve(const double* __restrict__ partial, int nblocks, int m, double pivot_tol,
                                 double* __restrict__ coef, int* __restrict__ accepted, const int* __restrict__ ctl) {
  if (ctl && ctl[0]) return;
  if (ctl) accepted += ctl[2];
  __shared__ double g[9];
  if (threadIdx.x < 9) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(size_t)b * 9 + threadIdx.x];
    g[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double A[3][3] = {{g[0], g[1], g[2]}, {g[1], g[3], g[4]}, {g[2], g[4], g[5]}};
  const double rhs[3] = {-g[6], -g[7], -g[8]};
  const int d = m - 1;
  double Lc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  bool ok = d > 0;
  for (int c = 0; c < d && ok; ++c) {
    double s = A[c][c];
    for (int j = 0; j < c; ++j) s -= Lc[c][j] * Lc[c][j];
    if (!(A[c][c] > 0.0) || !(s > pivot_tol * A[c][c])) {
      ok = false;
      break;
    }
    Lc[c][c] = sqrt(s);
    for (int i = c + 1; i < d; ++i) {
      double t = A[i][c];
      for (int j = 0; j < c; ++j) t -= Lc[i][j] * Lc[c][j];
      Lc[i][c] = t / Lc[c][c];
    }
  }
  double cf[4] = {0.0, 0.0, 0.0, 0.0};
  if (ok) {
    double y[3] = {0, 0, 0}, gam[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) {
      double t = rhs[i];
      for (int j = 0; j < i; ++j) t -= Lc[i][j] * y[j];
      y[i] = t / Lc[i][i];
    }
    for (int i = d - 1; i >= 0; --i) {
      double t = y[i];
      for (int j = i + 1; j < d; ++j) t -= Lc[j][i] * gam[j];
      gam[i] = t / Lc[i][i];
    }
    double sum = 0.0;
    for (int i = 0; i < d; ++i) {
      cf[i] = gam[i];
      sum += gam[i];
    }
    cf[d] = 1.0 - sum;
  } else {
    cf[d] = 1.0;
  }
  for (int i = 0; i < 4; ++i) coef[i] = cf[i];
  *accepted = ok ? 1 : 0;
}

cudaError_t launch_anderson_solve(const double* partial, int nblocks, int m, double pivot_tol, double* coef,
                                  int* accepted, cudaStream_t s, const int* ctl) {
  k_anderson_solve<<<1, 32, 0, s>>>(partial, nblocks, m, pivot_tol, coef, accepted, ctl);
  return cudaGetLastError();
}

template <typename T>
struct CombArgs {
  T* dst[3];
  T* bh[3];
  T* bl[3];
  const T* D[4][3];
  const T* uh[4][3];
  const T* ul[4][3];
};

// Dbar = sum_k c_k D_k; ubar = u_last + sum_{k<last} c_k (u_k - u_last) (the
// differences of nearby iterates are formed first, then added to u_last with
// an error-free sum when the low parts are present).  Every operand of an element is
// loaded before the first store, so that the loads of all three components are in
// flight together (the output arrays may alias nothing the compiler can see).
template <typename T, bool LO>
__global__ void k_combine(CombArgs<T> A, int m, const double* __restrict__ coef, long long count,
                          const int* __restrict__ stop) {
  if (stop && *stop) return;
  T c[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) c[j] = (j < m) ? (T)coef[j] : T(0);
  const int L = m - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    T Dv[3][4], Uh[3][4], Ul[3][4];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        Dv[q][j] = (j < m) ? __ldg(A.D[j][q] + i) : T(0);
        Uh[q][j] = (j < m) ? __ldg(A.uh[j][q] + i) : T(0);
        Ul[q][j] = (LO && j < m) ? __ldg(A.ul[j][q] + i) : T(0);
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) s += c[j] * Dv[q][j];
      T uL = Uh[q][0], lL = Ul[q][0];
#pragma unroll
      for (int j = 1; j < 4; ++j)
        if (j == L) {
          uL = Uh[q][j];
          lL = Ul[q][j];
        }
      T corr = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (j < L) {
          T dj = Uh[q][j] - uL;
          if (LO) dj += Ul[q][j] - lL;
          corr += c[j] * dj;
        }
      }
      A.dst[q][i] = s;
      if (LO) {
        const T s1 = uL + corr;
        const T bb = s1 - uL;
        const T e = (uL - (s1 - bb)) + (corr - bb);
        const T t = lL + e;
        const T h = s1 + t;
        A.bh[q][i] = h;
        A.bl[q][i] = t - (h - s1);
      } else {
        A.bh[q][i] = uL + corr;
      }
    }
  }
}

template <typename T>
cudaError_t launch_combine(T* const dst[3], T* const bh[3], T* const bl[3], const T* const D[4][3],
                           const T* const uh[4][3], const T* const ul[4][3], int m, const double* coef,
                           long long count, cudaStream_t s, const int* stop) {
  CombArgs<T> A;
  const bool lo = bl != nullptr && bl[0] != nullptr;
  for (int q = 0; q < 3; ++q) {
    A.dst[q] = dst[q];
    A.bh[q] = bh[q];
    A.bl[q] = lo ? bl[q] : nullptr;
    for (int j = 0; j < 4; ++j) {
      const int jj = j < m ? j : 0;
      A.D[j][q] = D[jj][q];
      A.uh[j][q] = uh[jj][q];
      A.ul[j][q] = lo ? ul[jj][q] : nullptr;
    }
  }
  if (lo) k_combine<T, true><<<152 * 8, 256, 0, s>>>(A, m, coef, count, stop);
  else k_combine<T, false><<<152 * 8, 256, 0, s>>>(A, m, coef, count, stop);
  return cudaGetLastError();
}

// ---- arithmetic peak probe --------------------------------------------------------------
// Eight independent chains of fused multiply-adds per thread (enough to cover the FMA
// latency), `iters` rounds; the result is written so the chains are not removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T t = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) t += x[k];
  if (t == T(-1.2345)) sink[blockIdx.x] = t;  // practically never: keeps the chains live
}

double fma_peak_flops(int fp64) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (sms > 0 ? sms : 152) * 8, threads = 256;
  const int iters = fp64 ? 4096 : 65536;
  void* sink = nullptr;
  if (cudaMalloc(&sink, blocks * sizeof(double)) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = -1.0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, 0);
    if (fp64) k_fma_peak<double><<<blocks, threads>>>((double*)sink, iters, 0.999999, 1e-7);
    else k_fma_peak<float><<<blocks, threads>>>((float*)sink, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f && rep > 0) {
      const double flops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
      if (flops > best) best = flops;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return cudaGetLastError() == cudaSuccess ? best : -1.0;
}

// Dense [q][z][y][x] <-> pitched component arrays.
template <typename T>
__global__ void k_pack(const T* s0, const T* s1, const T* s2, T* d0, T* d1, T* d2, T* dense, int N1, int N2, int N3,
                       long long sy, long long sz, int unpack) {
  const long long per = (long long)N1 * N2 * N3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * per;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / per);
    const long long r = i - q * per;
    const int x = (int)(r % N1);
    const long long r2 = r / N1;
    const int y = (int)(r2 % N2);
    const int z = (int)(r2 / N2);
    const long long off = x + y * sy + z * sz;
    if (unpack) {
      T* d = q == 0 ? d0 : (q == 1 ? d1 : d2);
      d[off] = dense[i];
    } else {
      const T* s = q == 0 ? s0 : (q == 1 ? s1 : s2);
      dense[i] = s[off];
    }
  }
}

template <typename T>
cudaError_t launch_pack(const T* const src[3], T* dst, int N1, int N2, int N3, long long sy, long long sz, int unpack,
                        cudaStream_t s) {
  // pack: src (pitched) -> dst (dense).  unpack: dst (dense) -> src (pitched, written through const_cast)
  T* p0 = const_cast<T*>(src[0]);
  T* p1 = const_cast<T*>(src[1]);
  T* p2 = const_cast<T*>(src[2]);
  k_pack<T><<<152 * 8, 256, 0, s>>>(src[0], src[1], src[2], p0, p1, p2, dst, N1, N2, N3, sy, sz, unpack);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_mask(T* f0, T* f1, T* f2, int l00, int l01, int l02, int h00, int h01, int h02, int l10, int l11,
                       int l12, int h10, int h11, int h12, int l20, int l21, int l22, int h20, int h21, int h22, int N1,
                       int N2, int N3, long long sy, long long sz) {
  const long long per = (long long)N1 * N2 * N3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % N1);
    const long long r2 = i / N1;
    const int y = (int)(r2 % N2);
    const int z = (int)(r2 / N2);
    const long long off = x + y * sy + z * sz;
    if (!(x >= l00 && x < h00 && y >= l01 && y < h01 && z >= l02 && z < h02)) f0[off] = T(0);
    if (!(x >= l10 && x < h10 && y >= l11 && y < h11 && z >= l12 && z < h12)) f1[off] = T(0);
    if (!(x >= l20 && x < h20 && y >= l21 && y < h21 && z >= l22 && z < h22)) f2[off] = T(0);
  }
}

template <typename T>
cudaError_t launch_mask(T* const f[3], const int lo[3][3], const int hi[3][3], int N1, int N2, int N3, long long sy,
                        long long sz, cudaStream_t s) {
  k_mask<T><<<152 * 8, 256, 0, s>>>(f[0], f[1], f[2], lo[0][0], lo[0][1], lo[0][2], hi[0][0], hi[0][1], hi[0][2],
                                    lo[1][0], lo[1][1], lo[1][2], hi[1][0], hi[1][1], hi[1][2], lo[2][0], lo[2][1],
                                    lo[2][2], hi[2][0], hi[2][1], hi[2][2], N1, N2, N3, sy, sz);
  return cudaGetLastError();
}

#define FFTM_INST(T)                                                                                               \
  template cudaError_t launch_copy_fields<T>(T* const[3], const T* const[3], long long, cudaStream_t);            \
  template cudaError_t launch_axpy_fields<T>(T* const[3], const T* const[3], const T* const[3], T, long long,     \
                                             cudaStream_t);                                                        \
  template cudaError_t launch_gram<T>(const T* const[4][3], int, long long, double*, int, cudaStream_t,           \
                                      const int*);                                                                 \
  template cudaError_t launch_combine<T>(T* const[3], T* const[3], T* const[3], const T* const[4][3],             \
                                         const T* const[4][3], const T* const[4][3], int, const double*,          \
                                         long long, cudaStream_t, const int*);                                     \
  template cudaError_t launch_pack<T>(const T* const[3], T*, int, int, int, long long, long long, int,            \
                                      cudaStream_t);                                                               \
  template cudaError_t launch_mask<T>(T* const[3], const int[3][3], const int[3][3], int, int, int, long long,    \
                                      long long, cudaStream_t);
FFTM_INST(float)
FFTM_INST(double)

}  // namespace fftm
