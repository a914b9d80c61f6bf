// Axis passes of the 3D transforms as dense contractions on the 5th-generation tensor
// cores (the "precision form": FP32 fields, BF16 operands, FP32 accumulation in TMEM).
//
// Every 1D transform of Table 1 and its inverse is a real L x L matrix T over the
// transform's node range (periodic axes in halfcomplex order).  A tile is 128 pencils of
// one component, staged once in shared memory as BF16.  y and z axes (pencils are the
// contiguous direction):
//     D[p][k] = sum_j S[p][j] T[k][j]
// with the tile S as the A operand (M = 128 pencils, MN-major) and T as the B operand
// (N = the padded output length, up to 256 per instruction), so TMEM lanes are pencils
// and a store writes 32 consecutive pencils.  x axis (pencils are rows of memory):
//     D[k][p] = sum_j T[k][j] S[p][j]
// with T as the A operand (M = outputs in blocks of 128) and S as the B operand (N = 128
// pencils, K-major), so TMEM lanes are outputs and a warp stores 32 consecutive nodes of
// one pencil row.  T arrives in 32-column chunks, laid out by the host in the exact
// core-matrix order, through a ring of shared-memory buffers filled by cp.async.bulk.
//
// Each CTA is persistent (one per SM) and warp-specialised: seven producer warps stage
// tiles into two operand buffers, one thread keeps the matrix ring filled ahead (across
// tile boundaries) and issues tcgen05.mma, and eight epilogue warps drain TMEM with
// tcgen05.ld; the roles hand over through mbarriers.  With Kp <= 256 a CTA keeps two
// accumulators, so the MMAs of one tile run while the previous one is drained.  The fused
// z pass multiplies the forward result by the Green factor, writes it back to shared
// memory as the A operand of a second contraction with the inverse matrix, and stores
// only the result.
//
// The transforms only precondition; convergence is decided on the FP32 residual of the
// stencil kernels, so BF16 rounding here changes the rate of the fixed point, not the
// field it converges to.
//
// Every wait (an mbarrier phase) is bounded: past the limit the CTA records an error in
// P.err, waits for its own copies and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "fftm_internal.cuh"
#include "fftm_umma.cuh"

namespace fftm {

constexpr int UM_P = 128;        // pencils per tile (MMA M on y and z, N on x)
constexpr int UM_KC = 32;        // K columns per matrix chunk (2 MMA k-steps)
// warp roles: 0-7 epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31), 8-14 stage pencil
// tiles, 15 streams the matrix chunks and issues the MMAs (lane 0)
constexpr int UM_EPI = 256;      // epilogue threads
constexpr int UM_PROD = 224;     // producer threads
constexpr int UM_THREADS = UM_EPI + UM_PROD + 32;
constexpr int UM_MAXBUF = 8;     // matrix chunk buffers at most
constexpr int UM_TMEM_COLS = 512;

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

// Shared-memory geometry of one CTA (bytes) for a padded transform length Kp (a multiple
// of 32).  x axis: the matrix is the A operand (M = outputs, padded to Mp = a multiple of
// 128) and the pencil tile the B operand (N = 128 pencils, K-major); y and z axes: the
// pencil tile is the A operand (M = 128 pencils, MN-major) and the matrix the B operand
// (N = outputs).  Matrices are streamed in chunks of 32 K columns through a ring of nbuf
// buffers.
struct UmGeom {
  uint32_t a_lbo, a_sbo, a_bytes;  // pencil tile
  uint32_t chunk_bytes;            // one matrix chunk (Mp x 32 BF16)
  int mp, nbuf;
  int acc_cols;                    // TMEM columns of one accumulator
  __host__ __device__ static UmGeom make(int Kp, int axis) {
    UmGeom g;
    g.mp = axis == 0 ? (Kp + 127) / 128 * 128 : Kp;
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
    g.a_bytes = (g.a_bytes + 1023) & ~1023u;
    g.chunk_bytes = (uint32_t)g.mp * UM_KC * 2;
    g.acc_cols = axis == 0 ? g.mp : Kp;  // x: Mp / 128 blocks of 128 pencils; y, z: Kp outputs
    const long long room = (long long)kMaxDynSmem - (long long)fixed_bytes(g.a_bytes);
    g.nbuf = room > 0 ? (int)(room / g.chunk_bytes) : 0;
    if (g.nbuf > UM_MAXBUF) g.nbuf = UM_MAXBUF;
    return g;
  }
  // two pencil-tile buffers, four tables of pencil row offsets (x pass), barriers and flags
  __host__ __device__ static size_t fixed_bytes(uint32_t a_bytes) { return 2 * (size_t)a_bytes + 4 * UM_P * 8 + 512; }
  __host__ __device__ size_t smem() const { return fixed_bytes(a_bytes) + (size_t)nbuf * chunk_bytes; }
};

__host__ __device__ inline UmGeom um_geom(int Kp, int axis) { return UmGeom::make(Kp, axis); }

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

// ---- producers --------------------------------------------------------------------------
// Stage one tile as BF16 (UM_PROD producer threads, ptid 0 .. UM_PROD - 1), sixteen (x) or
// eight (y, z) 16-byte loads in flight per thread.  x axis: the K index is j = x - xb with xb the range offset
// rounded down to a multiple of 4 (the host shifted the matrix columns by lo - xb), so each
// row is read with aligned 16-byte loads and the nodes outside the range are zeroed; the
// element offsets of the 128 pencil rows go to `offs` for the epilogue.  y and z: MN-major
// rows of 8 pencils.
template <int AXIS>
__device__ __forceinline__ void stage_tile(const TcPassParams& P, const Tile& T, const UmGeom& g, unsigned char* sA,
                                           long long* offs, int ptid) {
  const float* __restrict__ in = P.in[T.q];
  const int L = T.L, Kp = T.Kp, npen = T.npen;
  if (AXIS == 0) {
    // item (p, j4) covers the 4 nodes x = xb + j4 .. xb + j4 + 3 of pencil p; x is a
    // multiple of 4 below N1 and the row pitch a multiple of 8 >= N1, so the load stays in
    // the row.  Element (p, j) at (p>>3) SBO + (j>>3) LBO + (p&7) 16 + (j&7) 2.
    const long long sy = P.stride[1], sz = P.stride[2];
    const int N1 = P.N[0], N2 = P.N[1], lo = T.lo, xb = T.lo & ~3;
    if (ptid < UM_P) {
      const int r = T.row0 + ptid;
      offs[ptid] = ptid < npen ? (long long)(r % N2) * sy + (long long)(r / N2) * sz : 0;
    }
    const int nx4 = Kp / 4, total = UM_P * nx4;
    for (int i0 = ptid; i0 < total; i0 += 16 * UM_PROD) {
      float4 v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = i0 + u * UM_PROD;
        const int p = idx / nx4, x = xb + (idx % nx4) * 4;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < total && p < npen && x < N1) {
          const int r = T.row0 + p;
          v[u] = __ldg(reinterpret_cast<const float4*>(in + (long long)(r % N2) * sy + (long long)(r / N2) * sz + x));
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
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
    // item (pg, j) converts the 8 pencils 8 pg .. 8 pg + 7 of row j (32 aligned bytes: the
    // tile starts at a multiple of 8 and the row pitch is a multiple of 8)
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

// ---- the MMA thread ---------------------------------------------------------------------
// The contractions of a CTA, in issue order: C1(i) = forward matrix on tile i, C2(i) =
// inverse matrix on the Green-scaled tile i (fused pass).  With two accumulators the
// forward contraction of tile i + 1 is issued before C2(i), so that it runs while the
// epilogue applies the Green factor to tile i.
struct ContrSeq {
  int c1 = 0, c2 = 0;
  __device__ __forceinline__ void next(int fused, int nacc, int ntiles, int* tile, int* kind) {
    if (!fused) {
      *tile = c1++;
      *kind = 0;
    } else if (c1 < ntiles && c1 <= c2 + nacc - 1) {
      *tile = c1++;
      *kind = 0;
    } else {
      *tile = c2++;
      *kind = 1;
    }
  }
};

// Shared state of the CTA's barriers.
struct UmBars {
  uint64_t* a_full;     // [2]  UM_PROD arrivals: tile staged
  uint64_t* a_empty;    // [2]  1 (MMA commit): the tile's last contraction has read it
  uint64_t* acc_full;   // [2]  1 (MMA commit): a contraction into the accumulator is done
  uint64_t* acc_empty;  // [2]  UM_EPI arrivals: the epilogue has drained the accumulator
  uint64_t* a2_ready;   // 1    UM_EPI arrivals: Green-scaled tile written (fused)
  uint64_t* b_full;     // [UM_MAXBUF] transaction bytes: chunk landed
  uint64_t* b_empty;    // [UM_MAXBUF] 1 (MMA commit): chunk consumed
  uint64_t* done;       // 1    (MMA commit): every MMA of the CTA has completed
};

template <int AXIS, int FUSED>
__device__ void mma_thread(const TcPassParams& P, const UmGeom& g, unsigned char* const sA[2], unsigned char* sB,
                           const UmBars& B, uint32_t tmem, int nacc, int my_tiles, volatile int* abort) {
  const int ncontr = my_tiles * (FUSED ? 2 : 1);
  ContrSeq lseq, cseq;
  // loader position: contraction lt (tile lti, kind lk), chunk lc of lnch
  int lt = 0, lti = 0, lk = 0, lc = 0, lnch = 0;
  const unsigned char* lmat = nullptr;
  uint32_t lbytes = 0;
  // consumer position
  int ct = 0, cti = 0, ck = 0, cc = 0, cnch = 0, cstarted = 0;
  Tile CT;
  UmGeom cg = g;
  long long ni = 0, nc = 0;  // chunks issued, consumed
  long long idle = 0;
  auto load_contr = [&]() {
    lseq.next(FUSED, nacc, my_tiles, &lti, &lk);
    const Tile T = tile_of<AXIS, FUSED>(P, blockIdx.x + lti * gridDim.x);
    const UmGeom tg = um_geom(T.Kp, AXIS);
    lmat = reinterpret_cast<const unsigned char*>(lk ? P.A2[T.q] : P.A[T.q]);
    lbytes = tg.chunk_bytes;
    lnch = T.Kp / UM_KC;
    lc = 0;
  };
  auto cons_contr = [&]() {
    cseq.next(FUSED, nacc, my_tiles, &cti, &ck);
    CT = tile_of<AXIS, FUSED>(P, blockIdx.x + cti * gridDim.x);
    cg = um_geom(CT.Kp, AXIS);
    cnch = CT.Kp / UM_KC;
    cc = 0;
    cstarted = 0;
  };
  if (ncontr > 0) {
    load_contr();
    cons_contr();
  }
  while (ct < ncontr) {
    bool progress = false;
    // -- loader: the next chunk, once its ring buffer's previous chunk has been consumed
    if (lt < ncontr && ni < nc + g.nbuf) {
      const int b = (int)(ni % g.nbuf);
      const long long u = ni / g.nbuf;
      if (u == 0 || bar_test(&B.b_empty[b], (uint32_t)((u - 1) & 1))) {
        bulk_load(sB + (size_t)b * g.chunk_bytes, lmat + (size_t)lc * lbytes, lbytes, &B.b_full[b]);
        ++ni;
        progress = true;
        if (++lc == lnch && ++lt < ncontr) load_contr();
      }
    }
    // -- consumer: start the contraction once its operands and accumulator are free
    if (!cstarted) {
      const int s = cti & 1, a = cti % nacc;
      bool ready;
      if (ck == 0)
        ready = bar_test(&B.a_full[s], (uint32_t)((cti >> 1) & 1)) &&
                (cti < nacc || bar_test(&B.acc_empty[a], (uint32_t)(((cti / nacc) - 1) & 1)));
      else
        ready = bar_test(B.a2_ready, (uint32_t)(cti & 1));
      if (ready) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        cstarted = 1;
        progress = true;
      }
    }
    if (cstarted && nc < ni) {
      const int b = (int)(nc % g.nbuf);
      if (bar_test(&B.b_full[b], (uint32_t)((nc / g.nbuf) & 1))) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int s = cti & 1, a = cti % nacc;
        const uint32_t acc = tmem + (uint32_t)(a * 256);
        const uint32_t sb = smem_u32(sB + (size_t)b * g.chunk_bytes);
        const uint32_t sa = smem_u32(sA[s]);
#pragma unroll
        for (int st = 0; st < UM_KC / 16; ++st) {
          const int kk = cc * UM_KC + st * 16;
          const uint32_t accum = (cc > 0 || st > 0) ? 1u : 0u;
          if (AXIS == 0) {
            // D[m][p] += T[m][k] S[p][k]: A = matrix chunk (K-major, M blocks of 128 rows),
            // B = pencil tile (K-major, N = 128)
            const uint64_t db = smem_desc(sa + (uint32_t)(kk / 8) * cg.a_lbo, cg.a_lbo, cg.a_sbo);
            for (int mb = 0; mb < cg.mp / 128; ++mb) {
              const uint64_t da = smem_desc(sb + (uint32_t)mb * 16 * 512 + st * 256, 128, 512);
              mma_issue(acc + mb * 128, da, db, instr_desc(UM_P, false), accum);
            }
          } else {
            // D[p][k] += S[p][j] T[k][j]: A = pencil tile (MN-major; K-major for the Green-scaled
            // tile of C2), B = matrix chunk (K-major, N = outputs in blocks of up to 256)
            const bool mn = ck == 0;
            const uint32_t albo = mn ? cg.a_lbo : 128u, asbo = mn ? cg.a_sbo : (uint32_t)(CT.Kp / 8) * 128;
            const uint64_t da = smem_desc(sa + (uint32_t)(kk / 8) * albo, albo, asbo);
            for (int n0 = 0; n0 < CT.Kp; n0 += 256) {
              const int nn = CT.Kp - n0 < 256 ? CT.Kp - n0 : 256;
              const uint64_t db = smem_desc(sb + (uint32_t)(n0 / 8) * 512 + st * 256, 128, 512);
              mma_issue(acc + n0, da, db, instr_desc(nn, mn), accum);
            }
          }
        }
        mma_commit(&B.b_empty[b]);
        ++nc;
        progress = true;
        if (++cc == cnch) {
          mma_commit(&B.acc_full[a]);
          if (!FUSED || ck == 1) mma_commit(&B.a_empty[s]);
          if (++ct < ncontr) cons_contr();
        }
      }
    }
    if (progress) {
      idle = 0;
    } else if (++idle > 64) {
      __nanosleep(64);
      if (idle > UM_SPIN || ((idle & 255) == 0 && *abort)) {
        *abort = 1;
        break;
      }
    }
  }
  // copies still in flight (only after an abort) land, and every MMA completes, before the
  // CTA frees its TMEM and exits
  for (long long k = nc; k < ni; ++k) {
    const int b = (int)(k % g.nbuf);
    for (long long it = 0; it < UM_SPIN && !bar_test(&B.b_full[b], (uint32_t)((k / g.nbuf) & 1)); ++it)
      __nanosleep(64);
  }
  if (nc > 0) {
    mma_commit(B.done);
    for (long long it = 0; it < UM_SPIN && !bar_test(B.done, 0u); ++it) __nanosleep(64);
  }
}

// ---- the epilogue -----------------------------------------------------------------------
// UM_EPI threads, warps 0-7: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 and takes
// half h = w / 4 of the accumulator's columns (x: of its M blocks).
template <int AXIS>
__device__ __forceinline__ void store_tile(const TcPassParams& P, const Tile& T, uint32_t acc, const long long* offs,
                                           int warp, int lane) {
  const int q = T.q, L = T.L, Kp = T.Kp, npen = T.npen;
  float* __restrict__ out = P.out[q];
  const float sc = P.scale[q];
  const int gq = warp & 3, h = warp >> 2;
  const uint32_t lane_base = (uint32_t)(gq * 32) << 16;
  if (AXIS == 0) {
    // lanes are outputs: M index m <-> node x = xb + m; a warp writes 32 consecutive nodes of
    // one pencil row per store
    const float* __restrict__ bh = P.base[q];
    const float* __restrict__ bl = P.base_lo[q];
    float* __restrict__ ol = P.out_lo[q];
    const int mp = (Kp + 127) / 128 * 128, xb = T.lo & ~3;
    for (int mb = h; mb < mp / 128; mb += 2) {
      const int x = xb + mb * 128 + gq * 32 + lane;
      const bool ok = x >= T.lo && x < T.lo + L;
      if (bh == nullptr) {
        for (int p0 = 0; p0 < npen; p0 += 32) {
          float v[32];
          tmem_ld32(acc + lane_base + (uint32_t)(mb * 128 + p0), v);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (ok && p0 + u < npen) out[offs[p0 + u] + x] = sc * v[u];
        }
      } else {
        // the base values of the next 16 pencils are loaded while this chunk is summed
        float a0[16], b0[16], a1[16], b1[16];
        auto load_base = [&](int p0, float (&aa)[16], float (&bb)[16]) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const bool live = ok && p0 + u < npen;
            const long long at = offs[(p0 + u) & (UM_P - 1)] + x;
            aa[u] = live ? bh[at] : 0.f;
            bb[u] = (live && ol) ? bl[at] : 0.f;
          }
        };
        auto sum_store = [&](int p0, const float (&aa)[16], const float (&bb)[16]) {
          float v[16];
          tmem_ld16(acc + lane_base + (uint32_t)(mb * 128 + p0), v);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (!(ok && p0 + u < npen)) continue;
            const long long at = offs[p0 + u] + x;
            const float val = sc * v[u];
            if (ol == nullptr) {
              out[at] = aa[u] + val;
            } else {  // (hi, lo) = (bh, bl) + val with an error-free sum of the high parts
              const float s1 = aa[u] + val;
              const float bs = s1 - aa[u];
              const float er = (aa[u] - (s1 - bs)) + (val - bs);
              const float tt = bb[u] + er;
              const float hsum = s1 + tt;
              out[at] = hsum;
              ol[at] = tt - (hsum - s1);
            }
          }
        };
        load_base(0, a0, b0);
        for (int p0 = 0; p0 < npen; p0 += 32) {
          if (p0 + 16 < npen) load_base(p0 + 16, a1, b1);
          sum_store(p0, a0, b0);
          if (p0 + 16 >= npen) break;
          if (p0 + 32 < npen) load_base(p0 + 32, a0, b0);
          sum_store(p0 + 16, a1, b1);
        }
      }
    }
  } else {
    // lanes are pencils (consecutive in memory): one coalesced store per output
    const int p = gq * 32 + lane;
    const bool live = p < npen;
    const long long rowbase = T.base0 + p + (long long)T.lo * T.estride;
    const int half = Kp / 2;  // a multiple of 16
    int c0 = h * half;
    for (; c0 + 32 <= (h + 1) * half; c0 += 32) {
      float v[32];
      tmem_ld32(acc + lane_base + (uint32_t)c0, v);  // warp-collective: every lane takes part
      if (!live) continue;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int k = c0 + i;
        if (k < L) out[rowbase + (long long)k * T.estride] = sc * v[i];
      }
    }
    if (c0 < (h + 1) * half) {
      float v[16];
      tmem_ld16(acc + lane_base + (uint32_t)c0, v);
      if (live) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = c0 + i;
          if (k < L) out[rowbase + (long long)k * T.estride] = sc * v[i];
        }
      }
    }
  }
}

// Fused z pass: Green factor on (kx, ky, kz) of the forward result, written back K-major as
// the A operand of the inverse contraction.
__device__ __forceinline__ void green_tile(const TcPassParams& P, const Tile& T, uint32_t acc, unsigned char* sA,
                                           int warp, int lane) {
  const int gq = warp & 3, h = warp >> 2;
  const uint32_t lane_base = (uint32_t)(gq * 32) << 16;
  const int p = gq * 32 + lane;
  const int ky = T.yfix - P.flo[T.q][1];
  const int kx = T.x0 + p - P.flo[T.q][0];
  const bool live = p < T.npen && kx >= 0 && kx < P.fL[T.q][0];
  const uint32_t sbo2 = (uint32_t)(T.Kp / 8) * 128;
  const GreenLine G = tc_green_line(P, T.q, live ? kx : 0, ky);
  const float* __restrict__ Sz = P.S2[T.q][2];
  const float* __restrict__ Cz = P.C2[T.q][2];
  const int half = T.Kp / 2;
  for (int c0 = h * half; c0 < (h + 1) * half; c0 += 16) {
    // the z factors of these 16 outputs (the same for every lane) are loaded first, so that
    // their latency overlaps the TMEM load
    float sz[16], cz[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = min(c0 + u, T.L - 1);
      sz[u] = __ldg(Sz + k);
      cz[u] = __ldg(Cz + k);
    }
    float v[16];
    tmem_ld16(acc + lane_base + (uint32_t)c0, v);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = c0 + u;
      v[u] = (live && k < T.L) ? v[u] * G.at(sz[u], cz[u]) : 0.f;
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint4 w;
      w.x = pack_bf16x2(v[8 * hh + 0], v[8 * hh + 1]);
      w.y = pack_bf16x2(v[8 * hh + 2], v[8 * hh + 3]);
      w.z = pack_bf16x2(v[8 * hh + 4], v[8 * hh + 5]);
      w.w = pack_bf16x2(v[8 * hh + 6], v[8 * hh + 7]);
      *reinterpret_cast<uint4*>(sA + (uint32_t)(p >> 3) * sbo2 + (uint32_t)((c0 >> 3) + hh) * 128 + (p & 7) * 16) = w;
    }
  }
}

template <int AXIS, int FUSED>
__global__ void __launch_bounds__(UM_THREADS, 1) k_pass_umma(TcPassParams P, int maxKp) {
  if (P.stop && *P.stop) return;  // before any TMEM allocation or barrier
  extern __shared__ __align__(1024) unsigned char smem[];
  const UmGeom g = um_geom(maxKp, AXIS);
  unsigned char* const sA[2] = {smem, smem + g.a_bytes};
  // pencil row offsets of tile i (x pass) in table i % 4: the producers of tile i + 4 start
  // only after the epilogue of tile i has finished with it (through the accumulator hand-over)
  long long* offs_all = reinterpret_cast<long long*>(smem + 2 * (size_t)g.a_bytes);  // [4][UM_P]
  uint64_t* bars = reinterpret_cast<uint64_t*>(offs_all + 4 * UM_P);
  UmBars B;
  B.a_full = bars;
  B.a_empty = bars + 2;
  B.acc_full = bars + 4;
  B.acc_empty = bars + 6;
  B.a2_ready = bars + 8;
  B.b_full = bars + 9;
  B.b_empty = bars + 9 + UM_MAXBUF;
  B.done = bars + 9 + 2 * UM_MAXBUF;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 10 + 2 * UM_MAXBUF);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  unsigned char* sB = smem + UmGeom::fixed_bytes(g.a_bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = total_tiles<AXIS, FUSED>(P);
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nacc = 2 * g.acc_cols <= UM_TMEM_COLS ? 2 : 1;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(UM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      bar_init(&B.a_full[i], UM_PROD);
      bar_init(&B.a_empty[i], 1);
      bar_init(&B.acc_full[i], 1);
      bar_init(&B.acc_empty[i], UM_EPI);
    }
    bar_init(B.a2_ready, UM_EPI);
    bar_init(B.done, 1);
    for (int b = 0; b < UM_MAXBUF; ++b) {
      bar_init(&B.b_full[b], 1);
      bar_init(&B.b_empty[b], 1);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp >= UM_EPI / 32 && warp < (UM_EPI + UM_PROD) / 32) {
    // ---- producers: stage tile i into buffer i % 2 once the last contraction of tile i - 2
    // has read it ----
    const int ptid = tid - UM_EPI;
    for (int i = 0; i < my_tiles; ++i) {
      const int s = i & 1;
      if (i >= 2 && !bar_wait(&B.a_empty[s], ((i >> 1) - 1) & 1, abort)) break;
      const Tile T = tile_of<AXIS, FUSED>(P, blockIdx.x + i * gridDim.x);
      stage_tile<AXIS>(P, T, um_geom(T.Kp, AXIS), sA[s], offs_all + (i & 3) * UM_P, ptid);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      bar_arrive(&B.a_full[s]);
    }
  } else if (warp == (UM_EPI + UM_PROD) / 32) {
    // ---- MMA warp: lane 0 streams the matrix chunks and issues the MMAs ----
    if (lane == 0) mma_thread<AXIS, FUSED>(P, g, sA, sB, B, tmem, nacc, my_tiles, abort);
    __syncwarp();
  } else {
    // ---- epilogue warps 0-7 ----
    uint32_t acc_uses[2] = {0u, 0u};
    for (int i = 0; i < my_tiles; ++i) {
      const int s = i & 1, a = i % nacc;
      const uint32_t acc = tmem + (uint32_t)(a * 256);
      const Tile T = tile_of<AXIS, FUSED>(P, blockIdx.x + i * gridDim.x);
      if (!bar_wait(&B.acc_full[a], acc_uses[a] & 1, abort)) break;
      ++acc_uses[a];
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (FUSED) {
        green_tile(P, T, acc, sA[s], warp, lane);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        bar_arrive(B.a2_ready);
        if (!bar_wait(&B.acc_full[a], acc_uses[a] & 1, abort)) break;
        ++acc_uses[a];
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      }
      store_tile<AXIS>(P, T, acc, offs_all + (i & 3) * UM_P, warp, lane);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      bar_arrive(&B.acc_empty[a]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UM_TMEM_COLS));
}

template <int AXIS, int FUSED>
static cudaError_t launch_tc_one(const TcPassParams& P, int maxKp, cudaStream_t s) {
  const size_t smem = um_geom(maxKp, AXIS).smem();
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
    if (!pass_tc_fits(P.Kp[q], P.axis)) return cudaErrorInvalidValue;
    maxKp = maxKp > P.Kp[q] ? maxKp : P.Kp[q];
  }
  if (P.fused) {
    if (P.axis != 2) return cudaErrorInvalidValue;
    return launch_tc_one<2, 1>(P, maxKp, s);
  }
  if (P.axis == 0) return launch_tc_one<0, 0>(P, maxKp, s);
  if (P.axis == 1) return launch_tc_one<1, 0>(P, maxKp, s);
  return launch_tc_one<2, 0>(P, maxKp, s);
}

bool pass_tc_fits(int Kp, int axis) {
  if (Kp < UM_KC || Kp % UM_KC != 0) return false;
  const UmGeom g = um_geom(Kp, axis);
  // the accumulator (x: Mp / 128 blocks of 128 columns; y, z: Kp columns) fits TMEM, and at
  // least two matrix chunks fit beside the two pencil tiles
  return g.acc_cols <= UM_TMEM_COLS && g.nbuf >= 2 && g.smem() <= (size_t)kMaxDynSmem;
}

// Rows of the x-axis matrices (M padded to a multiple of 128); the y and z matrices have Kp.
int pass_tc_rows(int Kp, int axis) { return um_geom(Kp, axis).mp; }

}  // namespace fftm
