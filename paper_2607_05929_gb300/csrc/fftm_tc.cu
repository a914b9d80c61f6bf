// Axis passes of the 3D transforms as dense contractions on the tensor cores
// (the "precision form": FP32 fields, BF16 operands, FP32 accumulation).
//
// Every 1D transform of Table 1 and its inverse is a real L x L matrix over
// the transform's node range (periodic axes in halfcomplex order).  A pass
// computes, for a tile of TP pencils staged in shared memory as S[j][p],
//     C[k][p] = sum_j A[k][j] S[j][p]
// with mma.sync m16n8k16 (BF16 x BF16 -> FP32).  A (the matrix, padded to
// Kp x Kp with zeros, BF16, row-major) is read from global memory (it stays in
// L2); the B fragments are packed from S on the fly.  The fused z pass keeps
// C in registers, multiplies it by the Green factor, writes it back to S and
// contracts it with the inverse matrix.
//
// The transforms only apply the preconditioner (the Green operator); whether a
// load step has converged is decided on the residual D, computed in FP32 by
// the stencil kernels, so BF16 rounding here changes the rate of the fixed
// point, not the field it converges to.
#include <cuda_bf16.h>

#include "fftm_internal.cuh"

namespace fftm {

constexpr int TC_TP = 32;     // pencils per CTA
constexpr int TC_SP = 36;     // staging row pitch (== 4 mod 32: conflict-free B fragments)
constexpr int TC_WARPS = 8;   // m-tiles w, w + 8, w + 16 per warp
constexpr int TC_MAXMT = 3;   // so Kp <= 16 * 8 * 3 = 384

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// acc[mi][nt][e]: m-tile mt = warp + 8 mi, n-tile nt (8 pencils), element e of
// the m16n8 C fragment: e = 0 (row g, col 2t), 1 (g, 2t+1), 2 (g+8, 2t), 3 (g+8, 2t+1).
__device__ __forceinline__ void tc_gemm(const uint16_t* __restrict__ A, int Kp, const float* S,
                                        float acc[TC_MAXMT][4][4]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int MT = Kp >> 4;
#pragma unroll
  for (int mi = 0; mi < TC_MAXMT; ++mi)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mi][nt][e] = 0.f;
  const uint32_t* A32 = reinterpret_cast<const uint32_t*>(A);
  const int kp2 = Kp >> 1;  // row pitch in bf16 pairs
  for (int ks = 0; ks < MT; ++ks) {
    uint32_t b[4][2];
    const int r0 = ks * 16 + 2 * t;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + g;
      b[nt][0] = pack_bf16x2(S[r0 * TC_SP + col], S[(r0 + 1) * TC_SP + col]);
      b[nt][1] = pack_bf16x2(S[(r0 + 8) * TC_SP + col], S[(r0 + 9) * TC_SP + col]);
    }
#pragma unroll
    for (int mi = 0; mi < TC_MAXMT; ++mi) {
      const int mt = warp + TC_WARPS * mi;
      if (mt < MT) {
        const int row = mt * 16 + g;
        const int cp = ks * 8 + t;  // pair index of column ks*16 + 2t
        uint32_t a[4];
        a[0] = __ldg(A32 + row * kp2 + cp);
        a[1] = __ldg(A32 + (row + 8) * kp2 + cp);
        a[2] = __ldg(A32 + row * kp2 + cp + 4);
        a[3] = __ldg(A32 + (row + 8) * kp2 + cp + 4);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mi][nt], a, b[nt]);
      }
    }
  }
}

__device__ __forceinline__ float tc_green(const TcPassParams& P, int q, int kx, int ky, int kz) {
  const float sx = P.S2[q][0][kx], cx = P.C2[q][0][kx];
  const float sy = P.S2[q][1][ky], cy = P.C2[q][1][ky];
  const float sz = P.S2[q][2][kz], cz = P.C2[q][2][kz];
  float a0 = P.hf[0] * sx * cy * cz, a1 = P.hf[1] * cx * sy * cz, a2 = P.hf[2] * cx * cy * sz;
  if (P.tetra) {
    a0 += P.hf[0] * cx * sy * sz;
    a1 += P.hf[1] * sx * cy * sz;
    a2 += P.hf[2] * sx * sy * cz;
  }
  const float aq = (q == 0) ? a0 : ((q == 1) ? a1 : a2);
  const float den = P.two_mu0 * (a0 + a1 + a2) + P.lam0 * aq;
  return den > 0.f ? -P.gscale[q] / den : 0.f;
}

template <int AXIS, int FUSED>
__global__ void __launch_bounds__(TC_WARPS * 32) k_pass_tc(TcPassParams P) {
  extern __shared__ __align__(16) float S[];  // [Kp][TC_SP]
  const int q = blockIdx.y;
  const int L = P.L[q], lo = P.lo[q], Kp = P.Kp[q];
  const int N1 = P.N[0], N2 = P.N[1];
  const long long sx = P.stride[0], sy = P.stride[1], sz = P.stride[2];
  long long base0 = 0, estride = 0;
  int npen = TC_TP, row0 = 0, x0 = 0, yfix = 0;
  if (AXIS == 0) {
    row0 = blockIdx.x * TC_TP;
    npen = min(TC_TP, N2 * P.N[2] - row0);
    estride = sx;
  } else {
    const int ntx = (N1 + TC_TP - 1) / TC_TP;
    x0 = (blockIdx.x % ntx) * TC_TP;
    const int other = blockIdx.x / ntx;
    npen = min(TC_TP, N1 - x0);
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
    const int ky = yfix - P.flo[q][1];
    if (ky < 0 || ky >= P.fL[q][1]) return;  // a y position outside the range holds zeros
  }
  auto gaddr = [&](int p, int j) -> long long {
    if (AXIS == 0) {
      const int r = row0 + p;
      return (long long)(r % N2) * sy + (long long)(r / N2) * sz + (long long)(lo + j) * estride;
    }
    return base0 + p * sx + (long long)(lo + j) * estride;
  };

  const float* __restrict__ in = P.in[q];
  for (int idx = threadIdx.x; idx < Kp * TC_TP; idx += blockDim.x) {
    int j, p;
    if (AXIS == 0) {
      j = idx % Kp;
      p = idx / Kp;
    } else {
      p = idx % TC_TP;
      j = idx / TC_TP;
    }
    float* dst = S + j * TC_SP + p;
    if (j < L && p < npen) cp_async_4(dst, in + gaddr(p, j));
    else *dst = 0.f;
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  float acc[TC_MAXMT][4][4];
  tc_gemm(P.A[q], Kp, S, acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int MT = Kp >> 4;

  if (FUSED) {
    const int ky = yfix - P.flo[q][1];
    __syncthreads();  // every warp has finished reading S
#pragma unroll
    for (int mi = 0; mi < TC_MAXMT; ++mi) {
      const int mt = warp + TC_WARPS * mi;
      if (mt >= MT) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = mt * 16 + g + ((e >> 1) << 3);
          const int p = nt * 8 + 2 * t + (e & 1);
          const int kx = x0 + p - P.flo[q][0];
          float v = 0.f;
          if (k < L && p < npen && kx >= 0 && kx < P.fL[q][0]) v = acc[mi][nt][e] * tc_green(P, q, kx, ky, k);
          S[k * TC_SP + p] = v;
        }
    }
    __syncthreads();
    tc_gemm(P.A2[q], Kp, S, acc);
  }

  // ---- store ----
  float* __restrict__ out = P.out[q];
  const float* __restrict__ bh = P.base[q];
  const float* __restrict__ bl = P.base_lo[q];
  float* __restrict__ ol = P.out_lo[q];
  const float sc = P.scale[q];
#pragma unroll
  for (int mi = 0; mi < TC_MAXMT; ++mi) {
    const int mt = warp + TC_WARPS * mi;
    if (mt >= MT) continue;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = mt * 16 + g + ((e >> 1) << 3);
        const int p = nt * 8 + 2 * t + (e & 1);
        if (k >= L || p >= npen) continue;
        const long long at = gaddr(p, k);
        const float v = sc * acc[mi][nt][e];
        if (bh == nullptr) {
          out[at] = v;
        } else if (ol == nullptr) {
          out[at] = bh[at] + v;
        } else {  // (hi, lo) = (bh, bl) + v with an error-free sum of the high parts
          const float a = bh[at];
          const float s1 = a + v;
          const float bb = s1 - a;
          const float er = (a - (s1 - bb)) + (v - bb);
          const float tt = bl[at] + er;
          const float h = s1 + tt;
          out[at] = h;
          ol[at] = tt - (h - s1);
        }
      }
  }
}

template <int AXIS, int FUSED>
static cudaError_t launch_tc_one(const TcPassParams& P, int maxKp, cudaStream_t s) {
  const size_t smem = (size_t)maxKp * TC_SP * sizeof(float);
  auto kern = k_pass_tc<AXIS, FUSED>;
  // one opt-in limit for every problem (the attribute is per function and shared by threads)
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if (AXIS == 0) grid.x = (unsigned)((P.N[1] * P.N[2] + TC_TP - 1) / TC_TP);
  else grid.x = (unsigned)(((P.N[0] + TC_TP - 1) / TC_TP) * (AXIS == 1 ? P.N[2] : P.N[1]));
  grid.y = 3;
  kern<<<grid, TC_WARPS * 32, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_pass_tc(const TcPassParams& P, cudaStream_t s) {
  int maxKp = 0;
  for (int q = 0; q < 3; ++q) maxKp = maxKp > P.Kp[q] ? maxKp : P.Kp[q];
  if (maxKp > 16 * TC_WARPS * TC_MAXMT) return cudaErrorInvalidValue;
  if (P.fused) {
    if (P.axis != 2) return cudaErrorInvalidValue;
    return launch_tc_one<2, 1>(P, maxKp, s);
  }
  if (P.axis == 0) return launch_tc_one<0, 0>(P, maxKp, s);
  if (P.axis == 1) return launch_tc_one<1, 0>(P, maxKp, s);
  return launch_tc_one<2, 0>(P, maxKp, s);
}

}  // namespace fftm
