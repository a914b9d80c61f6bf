// Axis passes of the 3D transforms as dense contractions on the 5th-generation tensor
// cores (the "precision form": FP32 fields, BF16 operands, FP32 accumulation in TMEM).
//
// Every 1D transform of Table 1 and its inverse is a real L x L matrix T over the
// transform's node range (periodic axes in halfcomplex order).  One CTA transforms a
// tile of 128 pencils of one component:
//     D[p][k] = sum_j S[p][j] T[k][j]
// with tcgen05.mma kind::f16 (M = 128 pencils, N = the padded output length, up to 256
// per instruction, K = 16): the pencil tile S is the A operand, staged once in shared
// memory as BF16 (K-major for the x axis, whose pencils are contiguous in memory;
// MN-major for the y and z axes, whose pencils are the contiguous direction), and T is
// the B operand, streamed through three shared-memory buffers in 32-column chunks that
// the host laid out in the exact core-matrix order (one linear asynchronous copy per
// chunk).  The accumulator D lives in TMEM (lanes = pencils, columns = outputs) and is
// read back with tcgen05.ld for the epilogue.  The fused z pass multiplies D by the
// Green factor, writes it back to shared memory as the A operand of a second
// contraction with the inverse matrix, and stores only the result.
//
// The transforms only precondition; convergence is decided on the FP32 residual of the
// stencil kernels, so BF16 rounding here changes the rate of the fixed point, not the
// field it converges to.
//
// Every wait (an mbarrier phase) is bounded: past the limit the CTA records an error in
// P.err, waits for its own copies, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "fftm_internal.cuh"

namespace fftm {

constexpr int UM_P = 128;        // pencils per CTA (MMA M)
constexpr int UM_KC = 32;        // K columns per matrix chunk (2 MMA k-steps)
constexpr int UM_THREADS = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, column half w / 4
constexpr int UM_NBUF = 3;       // matrix chunk buffers (two chunks in flight ahead of the MMAs)
constexpr int UM_TMEM_COLS = 512;
constexpr long long UM_SPIN = 1ll << 24;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4, leading (K-direction) byte offset >> 4,
// stride (M/N-direction) byte offset >> 4, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: F32 accumulator, BF16 A and B, A K- or MN-major,
// B K-major, N >> 3, M >> 4.
__device__ __forceinline__ uint32_t instr_desc(int n, bool a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(UM_P >> 4) << 24);
}

__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < UM_SPIN && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
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

// Shared-memory geometry of one CTA (bytes).  Kp = padded transform length (input and
// output), a multiple of 32.
struct UmGeom {
  uint32_t a_lbo, a_sbo, a_bytes;  // pencil tile (A operand)
  uint32_t b_bytes;                // one matrix chunk (Kp x 32)
  __host__ __device__ static UmGeom make(int Kp, int axis) {
    UmGeom g;
    if (axis == 0) {  // K-major: element (p, j) at (p>>3) SBO + (j>>3) LBO + (p&7) 16 + (j&7) 2
      g.a_lbo = 144;  // 128 + 16: consecutive core matrices along K fall on different banks
      g.a_sbo = (uint32_t)(Kp / 8) * 144;
    } else {  // MN-major: element (p, j) at (p>>3) SBO + (j>>3) LBO + (j&7) 16 + (p&7) 2
      g.a_lbo = 128;
      g.a_sbo = (uint32_t)(Kp / 8) * 128 + 16;  // + 16: 8 pencil groups on different banks
    }
    g.a_bytes = (UM_P / 8) * g.a_sbo;
    // the fused pass writes its second A operand K-major with LBO 128, SBO (Kp/8) 128
    const uint32_t fused_bytes = (uint32_t)(UM_P / 8) * (uint32_t)(Kp / 8) * 128;
    if (fused_bytes > g.a_bytes) g.a_bytes = fused_bytes;
    // the x-axis epilogue stages 32 outputs of the 128 pencils here (pitch 33 floats)
    if ((uint32_t)(UM_P * 33 * 4) > g.a_bytes) g.a_bytes = UM_P * 33 * 4;
    g.a_bytes = (g.a_bytes + 1023) & ~1023u;
    g.b_bytes = (uint32_t)Kp * UM_KC * 2;
    return g;
  }
  __host__ __device__ size_t smem() const { return (size_t)a_bytes + UM_NBUF * (size_t)b_bytes + 64; }
};

// One contraction over Kp: A operand at sA (descriptor strides a_lbo / a_sbo, K-major or
// MN-major), B chunks streamed from `mat` through UM_NBUF buffers at sB (chunk c in buffer
// c % UM_NBUF, loaded UM_NBUF - 1 chunks ahead of the MMAs that read it).  Every thread
// takes part in the copies; thread 0 issues the MMAs and commits chunk c to bars[c % UM_NBUF].
// `uses` counts the completed phases of each barrier across calls.  Returns false (for
// every thread) on a timed-out wait.
__device__ bool contract(const uint16_t* __restrict__ mat, int Kp, unsigned char* sA, uint32_t a_lbo,
                         uint32_t a_sbo, bool a_mn, unsigned char* sB, uint32_t b_stride, uint64_t* bars,
                         uint32_t uses[UM_NBUF], uint32_t tmem, int* err) {
  const int tid = threadIdx.x;
  const int nch = Kp / UM_KC;
  const uint32_t chunk_bytes = (uint32_t)Kp * UM_KC * 2;
  auto load_chunk = [&](int c) {
    const char* src = reinterpret_cast<const char*>(mat) + (size_t)c * chunk_bytes;
    unsigned char* dst = sB + (size_t)(c % UM_NBUF) * b_stride;
    for (uint32_t off = tid * 16; off < chunk_bytes; off += UM_THREADS * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst + off)), "l"(src + off)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int c = 0; c < UM_NBUF - 1; ++c) {
    if (c < nch) load_chunk(c);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");  // keep the group count uniform
  }
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    const int cn = c + UM_NBUF - 1;  // the chunk loaded in this round
    if (cn < nch) {
      const int b = cn % UM_NBUF;
      if (cn >= UM_NBUF) {  // the MMAs of chunk cn - UM_NBUF read buffer b
        if (!bar_wait(&bars[b], uses[b] & 1)) ok = false;
        uses[b] += 1;
      }
      if (ok) load_chunk(cn);
      else asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_group %0;\n" ::"n"(UM_NBUF - 1) : "memory");  // chunk c has landed
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sb = smem_u32(sB + (size_t)(c % UM_NBUF) * b_stride);
#pragma unroll
      for (int s = 0; s < UM_KC / 16; ++s) {
        const int kk = c * UM_KC + s * 16;  // K offset in the A operand
        const uint64_t da = smem_desc(smem_u32(sA) + (uint32_t)(kk / 8) * a_lbo, a_lbo, a_sbo);
        for (int n0 = 0; n0 < Kp; n0 += 256) {
          const int nn = Kp - n0 < 256 ? Kp - n0 : 256;
          // B chunk: element (k, jj) at (k>>3) 512 + (jj>>3) 128 + (k&7) 16 + (jj&7) 2
          const uint64_t db = smem_desc(sb + (uint32_t)(n0 / 8) * 512 + s * 256, 128, 512);
          mma_issue(tmem + n0, da, db, instr_desc(nn, a_mn), (c > 0 || s > 0) ? 1u : 0u);
        }
      }
      mma_commit(&bars[c % UM_NBUF]);
    }
  }
  if (ok) {
    // commits not yet waited for: the last min(nch, UM_NBUF) chunks
    for (int c = (nch > UM_NBUF ? nch - UM_NBUF : 0); c < nch; ++c) {
      const int b = c % UM_NBUF;
      if (!bar_wait(&bars[b], uses[b] & 1)) ok = false;
      uses[b] += 1;
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return ok;
}

template <int AXIS, int FUSED>
__global__ void __launch_bounds__(UM_THREADS, 1) k_pass_umma(TcPassParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int q = blockIdx.y;
  const int L = P.L[q], lo = P.lo[q], Kp = P.Kp[q];
  const UmGeom g = UmGeom::make(Kp, AXIS);
  unsigned char* sA = smem;
  unsigned char* sB = smem + g.a_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + (size_t)UM_NBUF * g.b_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + UM_NBUF);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N2 = P.N[1];
  const long long sy = P.stride[1], sz = P.stride[2];

  // ---- tile of pencils ----
  long long base0 = 0, estride = 1;
  int npen = UM_P, row0 = 0, x0 = 0, yfix = 0;
  if (AXIS == 0) {
    row0 = blockIdx.x * UM_P;
    npen = min(UM_P, N2 * P.N[2] - row0);
  } else {
    // pencils x in [xb, xe) of this component (zero outside its node range), tiles of 128
    // starting at a multiple of 8 so that 8 pencils are one aligned 32-byte run
    const int xb = P.flo[q][0] & ~7, xe = P.flo[q][0] + P.fL[q][0];
    const int ntx = (xe - xb + UM_P - 1) / UM_P;
    const int xt = blockIdx.x % ntx, other = blockIdx.x / ntx;
    if (other >= (AXIS == 1 ? P.N[2] : N2)) return;
    x0 = xb + xt * UM_P;
    npen = min(x0 + UM_P, xe) - x0;
    if (AXIS == 1) {
      base0 = x0 + (long long)other * sz;
      estride = sy;
    } else {
      yfix = other;
      base0 = x0 + (long long)other * sy;
      estride = sz;
    }
  }
  if (FUSED) {
    const int ky = yfix - P.flo[q][1];
    if (ky < 0 || ky >= P.fL[q][1]) return;  // outside the y range the field is zero
  }
  if (npen <= 0) return;

  // ---- TMEM and barriers ----
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(UM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0)
    for (int b = 0; b < UM_NBUF; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[b])));

  // ---- pencil tile -> BF16 A operand ----
  const float* __restrict__ in = P.in[q];
  if (AXIS == 0) {
    // K-major; one warp per pencil, lanes along j two at a time
    for (int p = warp; p < UM_P; p += UM_THREADS / 32) {
      const bool live = p < npen;
      const float* src = in;
      if (live) {
        const int r = row0 + p;
        src = in + (long long)(r % N2) * sy + (long long)(r / N2) * sz + lo;
      }
#pragma unroll 4
      for (int j = 2 * lane; j < Kp; j += 64) {
        const float a = (live && j < L) ? __ldg(src + j) : 0.f;
        const float b = (live && j + 1 < L) ? __ldg(src + j + 1) : 0.f;
        const uint32_t off = (uint32_t)(p >> 3) * g.a_sbo + (uint32_t)(j >> 3) * g.a_lbo + (p & 7) * 16 + (j & 7) * 2;
        *reinterpret_cast<uint32_t*>(sA + off) = pack_bf16x2(a, b);
      }
    }
  } else {
    // MN-major; each thread converts 8 consecutive pencils of one row j (32 aligned bytes)
#pragma unroll 4
    for (int idx = tid; idx < (UM_P / 8) * Kp; idx += UM_THREADS) {
      const int pg = idx % (UM_P / 8), j = idx / (UM_P / 8);
      const int p0 = pg * 8;
      float v[8];
      if (j < L && p0 + 8 <= npen) {
        const float4* s4 = reinterpret_cast<const float4*>(in + base0 + (long long)(lo + j) * estride + p0);
        const float4 a = __ldg(s4), b = __ldg(s4 + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          v[i] = (j < L && p0 + i < npen) ? __ldg(in + base0 + (long long)(lo + j) * estride + p0 + i) : 0.f;
      }
      uint4 w;
      w.x = pack_bf16x2(v[0], v[1]);
      w.y = pack_bf16x2(v[2], v[3]);
      w.z = pack_bf16x2(v[4], v[5]);
      w.w = pack_bf16x2(v[6], v[7]);
      const uint32_t off = (uint32_t)pg * g.a_sbo + (uint32_t)(j >> 3) * g.a_lbo + (j & 7) * 16;
      *reinterpret_cast<uint4*>(sA + off) = w;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  uint32_t uses[UM_NBUF];
  for (int b = 0; b < UM_NBUF; ++b) uses[b] = 0u;
  const int wq = warp & 3, half = warp >> 2;  // TMEM lane quarter, column half
  const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
  const int p = wq * 32 + lane;  // this thread's pencil in the epilogue (TMEM lane)
  const int ncol16 = Kp / 16, c16_begin = half * ((ncol16 + 1) / 2), c16_end = half ? ncol16 : (ncol16 + 1) / 2;

  bool ok = contract(P.A[q], Kp, sA, g.a_lbo, g.a_sbo, AXIS != 0, sB, g.b_bytes, bars, uses, tmem, P.err);

  if (FUSED && ok) {
    // ---- Green factor on (kx, ky, kz), written back K-major as the A operand of the inverse ----
    const int ky = yfix - P.flo[q][1];
    const int kx = x0 + p - P.flo[q][0];
    const bool live = p < npen && kx >= 0 && kx < P.fL[q][0];
    const uint32_t sbo2 = (uint32_t)(Kp / 8) * 128;
    for (int c16 = c16_begin; c16 < c16_end; ++c16) {
      const int c0 = c16 * 16;
      float v[16];
      tmem_ld16(tmem + lane_base + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = c0 + i;
        v[i] = (live && k < L) ? v[i] * tc_green(P, q, kx, ky, k) : 0.f;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint4 w;
        w.x = pack_bf16x2(v[8 * h + 0], v[8 * h + 1]);
        w.y = pack_bf16x2(v[8 * h + 2], v[8 * h + 3]);
        w.z = pack_bf16x2(v[8 * h + 4], v[8 * h + 5]);
        w.w = pack_bf16x2(v[8 * h + 6], v[8 * h + 7]);
        const uint32_t off = (uint32_t)(p >> 3) * sbo2 + (uint32_t)((c0 >> 3) + h) * 128 + (p & 7) * 16;
        *reinterpret_cast<uint4*>(sA + off) = w;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    ok = contract(P.A2[q], Kp, sA, 128, sbo2, false, sB, g.b_bytes, bars, uses, tmem, P.err);
  }

  // ---- epilogue: TMEM -> (scale, accumulate) -> global ----
  if (ok) {
    float* __restrict__ out = P.out[q];
    const float* __restrict__ bh = P.base[q];
    const float* __restrict__ bl = P.base_lo[q];
    float* __restrict__ ol = P.out_lo[q];
    const float sc = P.scale[q];
    auto put = [&](long long at, float val) {
      if (bh == nullptr) {
        out[at] = val;
      } else if (ol == nullptr) {
        out[at] = bh[at] + val;
      } else {  // (hi, lo) = (bh, bl) + val with an error-free sum of the high parts
        const float a = bh[at];
        const float s1 = a + val;
        const float bb = s1 - a;
        const float er = (a - (s1 - bb)) + (val - bb);
        const float tt = bl[at] + er;
        const float hsum = s1 + tt;
        out[at] = hsum;
        ol[at] = tt - (hsum - s1);
      }
    };
    if (AXIS == 0) {
      // pencils are rows of memory: stage 32 outputs of all 128 pencils in shared memory
      // (pitch 33 floats), then write each pencil's 32 outputs with one coalesced warp access
      float* slab = reinterpret_cast<float*>(smem);  // the operands are no longer read
      for (int s0 = 0; s0 < Kp; s0 += 32) {
        float v[16];
        tmem_ld16(tmem + lane_base + s0 + 16 * half, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) slab[p * 33 + 16 * half + i] = sc * v[i];
        __syncthreads();
        const int k = s0 + lane;
        for (int pp = warp; pp < npen; pp += UM_THREADS / 32) {
          const int r = row0 + pp;
          if (k < L) put((long long)(r % N2) * sy + (long long)(r / N2) * sz + lo + k, slab[pp * 33 + lane]);
        }
        __syncthreads();
      }
    } else {
      const bool live = p < npen;
      const long long rowbase = base0 + p + (long long)lo * estride;
      for (int c16 = c16_begin; c16 < c16_end; ++c16) {
        const int c0 = c16 * 16;
        float v[16];
        tmem_ld16(tmem + lane_base + c0, v);  // warp-collective: every lane takes part
        if (!live) continue;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = c0 + i;
          if (k < L) put(rowbase + (long long)k * estride, sc * v[i]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UM_TMEM_COLS));
}

template <int AXIS, int FUSED>
static cudaError_t launch_tc_one(const TcPassParams& P, int maxKp, cudaStream_t s) {
  const size_t smem = UmGeom::make(maxKp, AXIS).smem();
  auto kern = k_pass_umma<AXIS, FUSED>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if (AXIS == 0) {
    grid.x = (unsigned)((P.N[1] * P.N[2] + UM_P - 1) / UM_P);
  } else {
    int ntx = 0;
    for (int q = 0; q < 3; ++q) {
      const int xb = P.flo[q][0] & ~7, xe = P.flo[q][0] + P.fL[q][0];
      ntx = max(ntx, (xe - xb + UM_P - 1) / UM_P);
    }
    grid.x = (unsigned)(ntx * (AXIS == 1 ? P.N[2] : P.N[1]));
  }
  grid.y = 3;
  kern<<<grid, UM_THREADS, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_pass_tc(const TcPassParams& P, cudaStream_t s) {
  int maxKp = 0;
  for (int q = 0; q < 3; ++q) {
    if (P.Kp[q] % UM_KC != 0 || P.Kp[q] > 480) return cudaErrorInvalidValue;
    maxKp = maxKp > P.Kp[q] ? maxKp : P.Kp[q];
  }
  if (UmGeom::make(maxKp, P.axis).smem() > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  if (P.fused) {
    if (P.axis != 2) return cudaErrorInvalidValue;
    return launch_tc_one<2, 1>(P, maxKp, s);
  }
  if (P.axis == 0) return launch_tc_one<0, 0>(P, maxKp, s);
  if (P.axis == 1) return launch_tc_one<1, 0>(P, maxKp, s);
  return launch_tc_one<2, 0>(P, maxKp, s);
}

}  // namespace fftm
