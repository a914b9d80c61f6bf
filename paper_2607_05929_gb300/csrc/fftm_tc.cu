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
// chunk).  Each CTA is persistent (one per SM) and warp-specialised: four warps stage the
// next tile into a second operand buffer while the MMA warp contracts the current one
// and four epilogue warps drain the previous accumulator, handing over through mbarriers.  The accumulator D lives in TMEM (lanes = pencils, columns = outputs) and is
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
// warp roles: 0-3 epilogue (TMEM lanes 32 w .. 32 w + 31), 4-11 stage pencil tiles,
// 12 streams the matrix chunks and issues the MMAs (lane 0)
constexpr int UM_THREADS = 416;
constexpr int UM_PROD = 256;  // producer threads
constexpr int UM_NBUF = 3;       // matrix chunk buffers (two chunks in flight ahead of the MMAs)
constexpr int UM_TMEM_COLS = 512;
constexpr long long UM_SPIN = 1ll << 24;  // mbarrier polls before giving up (~1 s with the back-off)

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

// Bounded wait for the phase with the given parity: non-blocking polls, backing off with
// __nanosleep after the first 64, so a phase that never completes is given up after about
// UM_SPIN x 64 ns (~1 s); also gives up as soon as another role of the CTA has (*abort).
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  uint32_t done = 0;
  for (long long it = 0; it < UM_SPIN && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (!done && it >= 64) {
      __nanosleep(64);
      if ((it & 255) == 255 && *abort) return false;
    }
  }
  if (!done) *abort = 1;
  return done != 0;
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// named barrier among the 128 threads of one role (ids 1, 2; 0 is __syncthreads)
__device__ __forceinline__ void role_sync(int id) { asm volatile("bar.sync %0, 128;\n" ::"r"(id) : "memory"); }

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

// Green factor B0 (Sec. 2.6.3) along one z line: with (kx, ky) fixed the denominator
// 2 mu0 (a0 + a1 + a2) + lam0 a_q is alpha cz + beta sz (each a_i is a sum of monomials in
// the squared sines and cosines, linear in cz and sz), so a line costs two coefficients
// and, per element, two products and a reciprocal.  A monomial with a zero factor stays
// exactly zero in the coefficients, so the null denominators are still exact zeros.
struct GreenLine {
  float alpha, beta, g;
  __device__ __forceinline__ float at(float sz, float cz) const {
    const float den = fmaf(alpha, cz, beta * sz);
    return den > 0.f ? __fdividef(g, den) : 0.f;
  }
};

__device__ __forceinline__ GreenLine tc_green_line(const TcPassParams& P, int q, int kx, int ky) {
  const float sx = P.S2[q][0][kx], cx = P.C2[q][0][kx];
  const float sy = P.S2[q][1][ky], cy = P.C2[q][1][ky];
  // a0 = c00 cz + c01 sz, a1 = c10 cz + c11 sz, a2 = c20 cz + c21 sz
  const float t = P.tetra ? 1.f : 0.f;
  const float c00 = P.hf[0] * sx * cy, c01 = t * P.hf[0] * cx * sy;
  const float c10 = P.hf[1] * cx * sy, c11 = t * P.hf[1] * sx * cy;
  const float c20 = t * P.hf[2] * sx * sy, c21 = P.hf[2] * cx * cy;
  const float aqc = q == 0 ? c00 : (q == 1 ? c10 : c20);
  const float aqs = q == 0 ? c01 : (q == 1 ? c11 : c21);
  GreenLine G;
  G.alpha = P.two_mu0 * (c00 + c10 + c20) + P.lam0 * aqc;
  G.beta = P.two_mu0 * (c01 + c11 + c21) + P.lam0 * aqs;
  G.g = -P.gscale[q];
  return G;
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
  // two pencil-tile buffers (one staged while the other is contracted), UM_NBUF chunk buffers,
  // barriers and flags
  __host__ __device__ size_t smem() const { return 2 * (size_t)a_bytes + UM_NBUF * (size_t)b_bytes + 256; }
};

// ---- tiles ------------------------------------------------------------------------------
// A pass enumerates, over the three components, the tiles of 128 pencils it transforms:
// x axis: rows (y, z) of the whole grid; y, z axes: runs of 128 pencils along x within
// the component's x node range (starting at a multiple of 8), for every z (y pass) or y
// (z pass; the fused pass only the y positions of the component's y range).
struct Tile {
  int q, L, lo, Kp, npen, row0, x0, yfix;
  long long base0, estride;
};

template <int AXIS, int FUSED>
__device__ __forceinline__ int comp_tiles(const TcPassParams& P, int q, int* ntx_out) {
  if (AXIS == 0) {
    *ntx_out = 1;
    return (P.N[1] * P.N[2] + UM_P - 1) / UM_P;
  }
  const int xb = P.flo[q][0] & ~7, xe = P.flo[q][0] + P.fL[q][0];
  const int ntx = (xe - xb + UM_P - 1) / UM_P;
  *ntx_out = ntx;
  const int nother = FUSED ? P.fL[q][1] : (AXIS == 1 ? P.N[2] : P.N[1]);
  return ntx * nother;
}

template <int AXIS, int FUSED>
__device__ __forceinline__ Tile tile_of(const TcPassParams& P, int t) {
  Tile T;
  int q = 0, ntx = 1, nt = comp_tiles<AXIS, FUSED>(P, 0, &ntx);
  while (t >= nt && q < 2) {
    t -= nt;
    ++q;
    nt = comp_tiles<AXIS, FUSED>(P, q, &ntx);
  }
  T.q = q;
  T.L = P.L[q];
  T.lo = P.lo[q];
  T.Kp = P.Kp[q];
  T.row0 = T.x0 = T.yfix = 0;
  T.base0 = 0;
  T.estride = 1;
  if (AXIS == 0) {
    T.row0 = t * UM_P;
    T.npen = min(UM_P, P.N[1] * P.N[2] - T.row0);
  } else {
    const int xb = P.flo[q][0] & ~7, xe = P.flo[q][0] + P.fL[q][0];
    const int xt = t % ntx, o = t / ntx;
    const int other = FUSED ? P.flo[q][1] + o : o;
    T.x0 = xb + xt * UM_P;
    T.npen = min(T.x0 + UM_P, xe) - T.x0;
    if (AXIS == 1) {
      T.base0 = T.x0 + (long long)other * P.stride[2];
      T.estride = P.stride[1];
    } else {
      T.yfix = other;
      T.base0 = T.x0 + (long long)other * P.stride[1];
      T.estride = P.stride[2];
    }
  }
  return T;
}

template <int AXIS, int FUSED>
__device__ __forceinline__ int total_tiles(const TcPassParams& P) {
  int n = 0, ntx;
  for (int q = 0; q < 3; ++q) n += comp_tiles<AXIS, FUSED>(P, q, &ntx);
  return n;
}

// ---- the three roles ---------------------------------------------------------------------
// Stage one tile as the BF16 A operand (UM_PROD producer threads, ptid 0 .. UM_PROD - 1),
// eight 16-byte loads in flight per thread.  x axis: the K index is j = x - xb with xb the
// range offset rounded down to a multiple of 4 (the host shifted the matrix columns by
// lo - xb), so each row is read with aligned 16-byte loads and the nodes outside the range
// are zeroed; y and z: MN-major rows of 8 pencils.
template <int AXIS>
__device__ __forceinline__ void stage_tile(const TcPassParams& P, const Tile& T, const UmGeom& g, unsigned char* sA,
                                           int ptid) {
  const float* __restrict__ in = P.in[T.q];
  const int L = T.L, Kp = T.Kp, npen = T.npen;
  if (AXIS == 0) {
    // K-major: item (p, j4) covers the 4 nodes x = xb + j4 .. xb + j4 + 3 of pencil p; x is a
    // multiple of 4 below N1 and the row pitch a multiple of 8 >= N1, so the load stays in
    // the row.  Element (p, j) at (p>>3) SBO + (j>>3) LBO + (p&7) 16 + (j&7) 2.
    const long long sy = P.stride[1], sz = P.stride[2];
    const int N1 = P.N[0], N2 = P.N[1], lo = T.lo, xb = T.lo & ~3;
    const int nx4 = Kp / 4, total = UM_P * nx4;
    for (int i0 = ptid; i0 < total; i0 += 8 * UM_PROD) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = i0 + u * UM_PROD;
        const int p = idx / nx4, x = xb + (idx % nx4) * 4;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < total && p < npen && x < N1) {
          const int r = T.row0 + p;
          v[u] = __ldg(reinterpret_cast<const float4*>(in + (long long)(r % N2) * sy + (long long)(r / N2) * sz + x));
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = i0 + u * UM_PROD;
        if (idx >= total) break;
        const int p = idx / nx4, j = (idx % nx4) * 4, x = xb + j;
        const float a0 = (x >= lo && x < lo + L) ? v[u].x : 0.f;
        const float a1 = (x + 1 >= lo && x + 1 < lo + L) ? v[u].y : 0.f;
        const float a2 = (x + 2 >= lo && x + 2 < lo + L) ? v[u].z : 0.f;
        const float a3 = (x + 3 >= lo && x + 3 < lo + L) ? v[u].w : 0.f;
        uint2 w;
        w.x = pack_bf16x2(a0, a1);
        w.y = pack_bf16x2(a2, a3);
        *reinterpret_cast<uint2*>(sA + (uint32_t)(p >> 3) * g.a_sbo + (uint32_t)(j >> 3) * g.a_lbo + (p & 7) * 16 +
                                  (j & 7) * 2) = w;
      }
    }
  } else {
    // MN-major; item (pg, j) converts the 8 pencils 8 pg .. 8 pg + 7 of row j (32 aligned
    // bytes: the tile starts at a multiple of 8 and the row pitch is a multiple of 8)
    const int total = (UM_P / 8) * Kp;
    for (int i0 = ptid; i0 < total; i0 += 4 * UM_PROD) {
      float4 v[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = i0 + u * UM_PROD;
        const int pg = idx % (UM_P / 8), j = idx / (UM_P / 8), p0 = pg * 8;
        const float* row = in + T.base0 + (long long)(T.lo + j) * T.estride + p0;
        v[u][0] = v[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < total && j < L) {
          if (p0 + 8 <= npen) {
            v[u][0] = __ldg(reinterpret_cast<const float4*>(row));
            v[u][1] = __ldg(reinterpret_cast<const float4*>(row) + 1);
          } else {
            float t[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) t[i] = p0 + i < npen ? __ldg(row + i) : 0.f;
            v[u][0] = make_float4(t[0], t[1], t[2], t[3]);
            v[u][1] = make_float4(t[4], t[5], t[6], t[7]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = i0 + u * UM_PROD;
        if (idx >= total) break;
        const int pg = idx % (UM_P / 8), j = idx / (UM_P / 8);
        uint4 w;
        w.x = pack_bf16x2(v[u][0].x, v[u][0].y);
        w.y = pack_bf16x2(v[u][0].z, v[u][0].w);
        w.z = pack_bf16x2(v[u][1].x, v[u][1].y);
        w.w = pack_bf16x2(v[u][1].z, v[u][1].w);
        *reinterpret_cast<uint4*>(sA + (uint32_t)pg * g.a_sbo + (uint32_t)(j >> 3) * g.a_lbo + (j & 7) * 16) = w;
      }
    }
  }
}

// One contraction over Kp by the MMA warp: A operand at sA, B chunks streamed from `mat`
// through the UM_NBUF buffers at sB (loaded UM_NBUF - 1 chunks ahead by the 32 lanes;
// chunk c is committed to bbar[c % UM_NBUF], counted in buses[]).  Lane 0 issues the MMAs.
__device__ __forceinline__ bool mma_contract(const uint16_t* __restrict__ mat, int Kp, unsigned char* sA,
                                             uint32_t a_lbo, uint32_t a_sbo, bool a_mn, unsigned char* sB,
                                             uint32_t b_stride, uint64_t* bbar, uint32_t buses[UM_NBUF],
                                             uint32_t tmem, volatile int* abort, int lane) {
  const int nch = Kp / UM_KC;
  const uint32_t chunk_bytes = (uint32_t)Kp * UM_KC * 2;
  // copies of a chunk into buffer b may start once the MMAs that last read b completed
  auto load_chunk = [&](int c) -> bool {
    const int b = c % UM_NBUF;
    bool ok = true;
    if (buses[b] & 0x80000000u) {  // an un-waited commit on b
      ok = bar_wait(&bbar[b], buses[b] & 1, abort);
      buses[b] = (buses[b] + 1) & 0x7FFFFFFFu;
    }
    const char* src = reinterpret_cast<const char*>(mat) + (size_t)c * chunk_bytes;
    unsigned char* dst = sB + (size_t)b * b_stride;
    if (ok)
      for (uint32_t off = lane * 16; off < chunk_bytes; off += 32 * 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst + off)), "l"(src + off)
                     : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    return ok;
  };
  bool ok = true;
  for (int c = 0; c < UM_NBUF - 1; ++c) {
    if (c < nch) ok = load_chunk(c) && ok;
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int c = 0; c < nch && ok; ++c) {
    const int cn = c + UM_NBUF - 1;
    if (cn < nch) ok = load_chunk(cn) && ok;
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group %0;\n" ::"n"(UM_NBUF - 1) : "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncwarp();
    if (!ok) break;
    if (lane == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sb = smem_u32(sB + (size_t)(c % UM_NBUF) * b_stride);
#pragma unroll
      for (int s = 0; s < UM_KC / 16; ++s) {
        const int kk = c * UM_KC + s * 16;
        const uint64_t da = smem_desc(smem_u32(sA) + (uint32_t)(kk / 8) * a_lbo, a_lbo, a_sbo);
        for (int n0 = 0; n0 < Kp; n0 += 256) {
          const int nn = Kp - n0 < 256 ? Kp - n0 : 256;
          const uint64_t db = smem_desc(sb + (uint32_t)(n0 / 8) * 512 + s * 256, 128, 512);
          mma_issue(tmem + n0, da, db, instr_desc(nn, a_mn), (c > 0 || s > 0) ? 1u : 0u);
        }
      }
      mma_commit(&bbar[c % UM_NBUF]);
    }
    __syncwarp();
    buses[c % UM_NBUF] |= 0x80000000u;  // its commit is now pending
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  return ok;
}

// The epilogue (128 threads, warps 0-3; thread = TMEM lane = pencil p of the tile).
template <int AXIS>
__device__ __forceinline__ void store_tile(const TcPassParams& P, const Tile& T, uint32_t tmem, float* slab,
                                           int warp, int lane) {
  const int q = T.q, L = T.L, Kp = T.Kp, npen = T.npen;
  float* __restrict__ out = P.out[q];
  const float* __restrict__ bh = P.base[q];
  const float* __restrict__ bl = P.base_lo[q];
  float* __restrict__ ol = P.out_lo[q];
  const float sc = P.scale[q];
  const int p = warp * 32 + lane;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  if (AXIS == 0) {
    // pencils are rows of memory: stage 32 outputs of the 128 pencils (pitch 33 floats) and
    // write each pencil's 32 outputs with one coalesced warp access, 8 rows in flight
    const long long sy = P.stride[1], sz = P.stride[2];
    const int N2 = P.N[1];
    for (int s0 = 0; s0 < Kp; s0 += 32) {
      float v[16];
      tmem_ld16(tmem + lane_base + s0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) slab[p * 33 + i] = sc * v[i];
      tmem_ld16(tmem + lane_base + s0 + 16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) slab[p * 33 + 16 + i] = sc * v[i];
      role_sync(1);
      const int k = s0 + lane;
      if (k < L) {
        for (int pp0 = warp; pp0 < npen; pp0 += 4 * 8) {
          long long at[8];
          float a[8], b[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int pp = pp0 + 4 * u;
            const int r = T.row0 + (pp < npen ? pp : 0);
            at[u] = (long long)(r % N2) * sy + (long long)(r / N2) * sz + T.lo + k;
            a[u] = (bh && pp < npen) ? bh[at[u]] : 0.f;
            b[u] = (ol && pp < npen) ? bl[at[u]] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int pp = pp0 + 4 * u;
            if (pp >= npen) break;
            const float val = slab[pp * 33 + lane];
            if (bh == nullptr) {
              out[at[u]] = val;
            } else if (ol == nullptr) {
              out[at[u]] = a[u] + val;
            } else {  // (hi, lo) = (bh, bl) + val with an error-free sum of the high parts
              const float s1 = a[u] + val;
              const float bb = s1 - a[u];
              const float er = (a[u] - (s1 - bb)) + (val - bb);
              const float tt = b[u] + er;
              const float hsum = s1 + tt;
              out[at[u]] = hsum;
              ol[at[u]] = tt - (hsum - s1);
            }
          }
        }
      }
      role_sync(1);
    }
  } else {
    const bool live = p < npen;
    const long long rowbase = T.base0 + p + (long long)T.lo * T.estride;
    for (int c0 = 0; c0 < Kp; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + c0, v);  // warp-collective: every lane takes part
      if (!live) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = c0 + i;
        if (k < L) out[rowbase + (long long)k * T.estride] = sc * v[i];
      }
    }
  }
}

template <int AXIS, int FUSED>
__global__ void __launch_bounds__(UM_THREADS, 1) k_pass_umma(TcPassParams P, int maxKp) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const UmGeom g = UmGeom::make(maxKp, AXIS);
  unsigned char* sA[2] = {smem, smem + g.a_bytes};
  unsigned char* sB = smem + 2 * (size_t)g.a_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + (size_t)UM_NBUF * g.b_bytes);
  uint64_t* a_full = bars;          // [2], UM_PROD arrivals (producers)
  uint64_t* a_empty = bars + 2;     // [2], 128 arrivals (epilogue)
  uint64_t* acc_full = bars + 4;    // 1 arrival (MMA commit)
  uint64_t* acc_empty = bars + 5;   // 128 arrivals (epilogue)
  uint64_t* a2_ready = bars + 6;    // 128 arrivals (epilogue, fused pass)
  uint64_t* b_empty = bars + 7;     // [UM_NBUF], MMA commits
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7 + UM_NBUF);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = total_tiles<AXIS, FUSED>(P);
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(UM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    bar_init(&a_full[0], UM_PROD);
    bar_init(&a_full[1], UM_PROD);
    bar_init(&a_empty[0], 128);
    bar_init(&a_empty[1], 128);
    bar_init(acc_full, 1);
    bar_init(acc_empty, 128);
    bar_init(a2_ready, 128);
    for (int b = 0; b < UM_NBUF; ++b) bar_init(&b_empty[b], 1);
    *abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp >= 4 && warp < 4 + UM_PROD / 32) {
    // ---- producers: stage tile i into buffer i % 2 once the epilogue of tile i - 2 freed it ----
    const int ptid = tid - 128;
    for (int i = 0; i < my_tiles; ++i) {
      const int s = i & 1;
      if (i >= 2 && !bar_wait(&a_empty[s], ((i >> 1) - 1) & 1, abort)) break;
      const Tile T = tile_of<AXIS, FUSED>(P, blockIdx.x + i * gridDim.x);
      stage_tile<AXIS>(P, T, UmGeom::make(T.Kp, AXIS), sA[s], ptid);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      bar_arrive(&a_full[s]);
    }
  } else if (warp == 4 + UM_PROD / 32) {
    // ---- MMA warp ----
    uint32_t buses[UM_NBUF];
    for (int b = 0; b < UM_NBUF; ++b) buses[b] = 0u;
    for (int i = 0; i < my_tiles; ++i) {
      const int s = i & 1;
      if (!bar_wait(&a_full[s], (i >> 1) & 1, abort)) break;
      if (i >= 1 && !bar_wait(acc_empty, (i - 1) & 1, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const Tile T = tile_of<AXIS, FUSED>(P, blockIdx.x + i * gridDim.x);
      const UmGeom gt = UmGeom::make(T.Kp, AXIS);
      if (!mma_contract(P.A[T.q], T.Kp, sA[s], gt.a_lbo, gt.a_sbo, AXIS != 0, sB, g.b_bytes, b_empty, buses, tmem,
                        abort, lane))
        break;
      if (lane == 0) mma_commit(acc_full);
      __syncwarp();
      if (FUSED) {
        if (!bar_wait(a2_ready, i & 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!mma_contract(P.A2[T.q], T.Kp, sA[s], 128, (uint32_t)(T.Kp / 8) * 128, false, sB, g.b_bytes, b_empty,
                          buses, tmem, abort, lane))
          break;
        if (lane == 0) mma_commit(acc_full);
        __syncwarp();
      }
    }
    // commits still pending on the chunk buffers (they complete with the last acc_full)
    for (int b = 0; b < UM_NBUF; ++b)
      if (buses[b] & 0x80000000u) bar_wait(&b_empty[b], buses[b] & 1, abort);
  } else {
    // ---- epilogue warps 0-3 ----
    uint32_t acc_uses = 0;
    for (int i = 0; i < my_tiles; ++i) {
      const int s = i & 1;
      const Tile T = tile_of<AXIS, FUSED>(P, blockIdx.x + i * gridDim.x);
      if (!bar_wait(acc_full, acc_uses & 1, abort)) break;
      ++acc_uses;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
      const int p = warp * 32 + lane;
      if (FUSED) {
        // Green factor on (kx, ky, kz), written back K-major as the A operand of the inverse
        const int ky = T.yfix - P.flo[T.q][1];
        const int kx = T.x0 + p - P.flo[T.q][0];
        const bool live = p < T.npen && kx >= 0 && kx < P.fL[T.q][0];
        const uint32_t sbo2 = (uint32_t)(T.Kp / 8) * 128;
        const GreenLine G = tc_green_line(P, T.q, live ? kx : 0, ky);
        const float* __restrict__ Sz = P.S2[T.q][2];
        const float* __restrict__ Cz = P.C2[T.q][2];
        for (int c0 = 0; c0 < T.Kp; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + lane_base + c0, v);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int k = c0 + u;
            v[u] = (live && k < T.L) ? v[u] * G.at(Sz[k], Cz[k]) : 0.f;
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint4 w;
            w.x = pack_bf16x2(v[8 * h + 0], v[8 * h + 1]);
            w.y = pack_bf16x2(v[8 * h + 2], v[8 * h + 3]);
            w.z = pack_bf16x2(v[8 * h + 4], v[8 * h + 5]);
            w.w = pack_bf16x2(v[8 * h + 6], v[8 * h + 7]);
            *reinterpret_cast<uint4*>(sA[s] + (uint32_t)(p >> 3) * sbo2 + (uint32_t)((c0 >> 3) + h) * 128 +
                                      (p & 7) * 16) = w;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        bar_arrive(a2_ready);
        if (!bar_wait(acc_full, acc_uses & 1, abort)) break;
        ++acc_uses;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      }
      store_tile<AXIS>(P, T, tmem, reinterpret_cast<float*>(sA[s]), warp, lane);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      bar_arrive(acc_empty);
      bar_arrive(&a_empty[s]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UM_TMEM_COLS));
}

template <int AXIS, int FUSED>
static cudaError_t launch_tc_one(const TcPassParams& P, int maxKp, cudaStream_t s) {
  const size_t smem = UmGeom::make(maxKp, AXIS).smem();
  auto kern = k_pass_umma<AXIS, FUSED>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one persistent CTA per SM (each holds all 512 TMEM columns)
  kern<<<dim3((unsigned)(sms > 0 ? sms : 152)), UM_THREADS, smem, s>>>(P, maxKp);
  return cudaGetLastError();
}

cudaError_t launch_pass_tc(const TcPassParams& P, cudaStream_t s) {
  int maxKp = 0;
  for (int q = 0; q < 3; ++q) {
    if (P.Kp[q] % UM_KC != 0 || P.Kp[q] > 512) return cudaErrorInvalidValue;
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

bool pass_tc_fits(int Kp, int axis) {
  return Kp % UM_KC == 0 && Kp <= 512 && UmGeom::make(Kp, axis).smem() <= (size_t)kMaxDynSmem;
}

}  // namespace fftm
