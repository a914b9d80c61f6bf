// Axis passes of the 3D transforms as dense contractions on the 5th-generation tensor cores
// with TF32 operands: the FP32 fields and FP32 transform matrices are read as they are
// stored and multiplied by tcgen05.mma kind::tf32 (10-bit significands in the products,
// FP32 accumulation in TMEM).  The precision form of the transforms (Table 1 as dense
// matrices, Sec. 2.7.2); the residual that decides convergence stays in FP32.
//
// Every 1D transform of Table 1 and its inverse is a real L x L matrix T over the
// transform's node range (periodic axes in halfcomplex order).  A tile is 128 pencils of one
// component.  y and z axes (pencils are the contiguous direction):
//     D[p][k] = sum_j S[p][j] T[k][j]
// with the tile S as the A operand (M = 128 pencils) and T as the B operand (N = the padded
// output length, up to 256 per instruction), both K-major (the producers transpose 4 x 4
// blocks of the tile in registers); TMEM lanes are pencils and one store writes 32
// consecutive pencils.  x axis (pencils are rows of memory):
//     D[k][p] = sum_j T[k][j] S[p][j]
// with T as the A operand (M = outputs in blocks of 128) and S as the B operand (N = 128
// pencils, K-major); TMEM lanes are outputs and a warp stores 32 consecutive nodes of a row.
//
// The contraction dimension streams through a ring of shared-memory stages, each holding
// 32 K-columns of the tile (filled by seven producer warps with 16-byte cp.async copies, up to
// three stages in flight, then transposed in 4 x 4 blocks on y and z and rounded to the nearest
// TF32 in place) and of the matrix (one bulk copy, entries rounded to TF32 on the host).  One thread issues the MMAs
// of a stage as soon as both halves have landed and releases the stage when they have read
// it; eight epilogue warps drain the TMEM accumulators (two, alternating, when they fit)
// while the next tile is contracted.  Every wait is bounded: past the limit the CTA records
// an error in P.err, lets its copies and MMAs finish, frees its TMEM and returns.
#include <cudaTypedefs.h>

#include "fftm_internal.cuh"
#include "fftm_umma.cuh"

namespace fftm {

constexpr int TF_P = 128;      // pencils per tile
constexpr int TF_KC = 32;      // K columns per stage (four MMA k-steps of 8)
constexpr int TF_EPI = 256;    // epilogue threads (warps 0-7)
constexpr int TF_PROD = 224;   // producer threads (warps 8-14)
constexpr int TF_THREADS = TF_EPI + TF_PROD + 32;  // warp 15: matrix copies and MMAs (lane 0)
constexpr int TF_MAXST = 8;
constexpr int TF_TMEM_COLS = 512;
constexpr uint32_t TF_TILE_BYTES = TF_P * TF_KC * 4;

// Instruction descriptor, kind::tf32: F32 accumulator, TF32 A and B, both K-major,
// N >> 3, M >> 4.
__device__ __forceinline__ uint32_t tf_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TF_P >> 4) << 24);
}

// K-major operand with the 128-byte swizzle (rows of 128 bytes, 8-row atoms of 1024 bytes, the
// 16-byte chunks of row r at chunk ^ (r & 7)): the layout a TMA box of 32 FP32 x rows writes with
// CU_TENSOR_MAP_SWIZZLE_128B.  A k-step of 8 elements advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  return smem_desc(saddr, 16, 1024) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tf_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}


// Shared-memory geometry for Kn outputs on the tensor cores (a multiple of 32).  xtra: room for
// the partial sums of the one output that the producers contract (y, z, 257 outputs).
constexpr uint32_t TF_XBYTES = 2u * 8u * TF_P * 4u;  // two tiles x eight row groups x 128 pencils

struct TfGeom {
  int mp;            // matrix rows (x: Kn rounded up to 128; y, z: Kn)
  uint32_t stage;    // bytes of one stage: tile part, matrix part (mp x 32 FP32), raw part
  int nst;           // stages
  int acc_cols;      // TMEM columns of one accumulator
  int raw;           // y, z: the tile arrives by TMA in a raw part (rows of 128 pencils) and is
                     // transposed from there (when three stages still fit); else per-thread copies
  int xtra;          // the partial-sum area follows the stages
  __host__ __device__ static TfGeom make(int Kn, int axis, int xtra = 0) {
    TfGeom g;
    g.mp = axis == 0 ? (Kn + 127) / 128 * 128 : Kn;
    g.acc_cols = axis == 0 ? g.mp : Kn;
    g.xtra = xtra ? 1 : 0;
    const long long room = (long long)kMaxDynSmem - 2048 - (xtra ? (long long)TF_XBYTES : 0);
    for (g.raw = axis == 0 ? 0 : 1; g.raw >= 0; --g.raw) {
      g.stage = (TF_TILE_BYTES * (1u + (uint32_t)g.raw) + (uint32_t)g.mp * TF_KC * 4 + 1023u) & ~1023u;
      g.nst = (int)(room / g.stage);
      if (g.nst >= 3) break;
    }
    if (g.raw < 0) g.raw = 0;
    if (g.nst > TF_MAXST) g.nst = TF_MAXST;
    return g;
  }
  __host__ __device__ uint32_t raw_off() const { return TF_TILE_BYTES + (uint32_t)mp * TF_KC * 4; }
  __host__ __device__ uint32_t xoff() const { return (uint32_t)nst * stage; }  // from the first stage
  __host__ __device__ size_t smem() const { return 2048 + (size_t)nst * stage + (xtra ? TF_XBYTES : 0); }
};

// ---- tiles ------------------------------------------------------------------------------
// x axis: runs of 128 consecutive (y, z) rows of the whole grid; y and z axes: runs of 128
// pencils along x within the component's x node range (from a multiple of 8), for every z
// (y pass) or for every y of the component's y range (z passes).
struct TfTile {
  int q, L, lo, Kp, Kn, npen, row0, x0, other;
  int xt;  // the producers contract output 256 (Kn = 256, L = 257)
  long long base0, estride;
};

template <int AXIS>
__device__ __forceinline__ int tf_comp_tiles(const TfPassParams& P, int q, int* ntx_out) {
  if (AXIS == 0) {
    *ntx_out = 1;
    return (P.N[1] * P.N[2] + TF_P - 1) / TF_P;
  }
  const int xb = P.flo[q][0] & ~7, xe = P.flo[q][0] + P.fL[q][0];
  const int ntx = (xe - xb + TF_P - 1) / TF_P;
  *ntx_out = ntx;
  const int nother = AXIS == 1 ? P.N[2] : P.fL[q][1];
  return ntx * nother;
}

template <int AXIS>
__device__ __forceinline__ TfTile tf_tile_of(const TfPassParams& P, int t) {
  TfTile T;
  int q = 0, ntx = 1, nt = tf_comp_tiles<AXIS>(P, 0, &ntx);
  while (t >= nt && q < 2) {
    t -= nt;
    ++q;
    nt = tf_comp_tiles<AXIS>(P, q, &ntx);
  }
  T.q = q;
  T.L = P.L[q];
  T.lo = P.lo[q];
  T.Kp = P.Kp[q];
  T.Kn = P.Kn[q];
  T.xt = AXIS != 0 && P.xrow[q] != nullptr;
  T.row0 = T.x0 = T.other = 0;
  T.base0 = 0;
  T.estride = 1;
  if (AXIS == 0) {
    T.row0 = t * TF_P;
    T.npen = min(TF_P, P.N[1] * P.N[2] - T.row0);
  } else {
    const int xb = P.flo[q][0] & ~7, xe = P.flo[q][0] + P.fL[q][0];
    const int xt = t % ntx, o = t / ntx;
    T.other = AXIS == 1 ? o : P.flo[q][1] + o;
    T.x0 = xb + xt * TF_P;
    T.npen = min(T.x0 + TF_P, xe) - T.x0;
    T.base0 = T.x0 + (long long)T.other * (AXIS == 1 ? P.stride[2] : P.stride[1]);
    T.estride = AXIS == 1 ? P.stride[1] : P.stride[2];
  }
  return T;
}

template <int AXIS>
__device__ __forceinline__ int tf_total_tiles(const TfPassParams& P) {
  int n = 0, ntx;
  for (int q = 0; q < 3; ++q) n += tf_comp_tiles<AXIS>(P, q, &ntx);
  return n;
}

// ---- producers ---------------------------------------------------------------------------
// The tile part of a stage holds 128 rows (pencils) x 32 K values in the K-major core-matrix
// order: element (p, k) at (p>>3) 1024 + (k>>2) 128 + (p&7) 16 + (k&3) 4 bytes (LBO = 128
// along K, SBO = 1024 per 8 rows), zero where it falls outside the array or the tile.
// The producers fill it in two steps: 16-byte cp.async copies from global memory (zero-filled
// outside), several stages in flight per thread without holding registers, then, once a
// thread's copies of a stage have landed, an in-place pass over the cells it copied:
//  x axis: 1024 pieces (row p, group g) of 4 consecutive x land in their final cells; the pass
//    rounds them to the nearest TF32;
//  y, z axes: 256 blocks (pencil group pg, row group kq) of 4 pencils x 4 rows; row 4 kq + r of
//    pencils 4 pg .. 4 pg + 3 lands in the cell of pencil 4 pg + r, so the pass reads the
//    block's four cells, transposes them in registers (each pencil's 4 K values in one cell)
//    and writes them back rounded, to the same four cells.
constexpr int TF_XPC = 5;  // x axis: 16-byte pieces per producer thread and stage (1024 pieces, 224 threads)

constexpr int TF_BLK = 2;  // 4 x 4 blocks per producer thread and stage (256 blocks, 224 threads)

// FP32 -> the nearest TF32 value (ties away from zero), kept in an FP32 register
__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

// waits until at most n of this thread's copy groups are still in flight (n <= 3)
__device__ __forceinline__ void cp_async_wait(int n) {
  if (n <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else if (n == 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
  else asm volatile("cp.async.wait_group 3;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t tf_cell(int p, int kq) {
  return (uint32_t)(p >> 3) * 1024u + (uint32_t)kq * 128u + (uint32_t)(p & 7) * 16u;
}

template <int AXIS>
__device__ __forceinline__ void tf_issue(const TfPassParams& P, const TfTile& T, int c, int ptid, uint32_t sdst) {
  const float* __restrict__ in = P.in[T.q];
  const long long PX = P.stride[1];  // row pitch (a multiple of 8, >= N1)
  if (AXIS == 0) {
    const int N2 = P.N[1];
    const long long sy = P.stride[1], sz = P.stride[2];
    const int xb = T.lo & ~3;
#pragma unroll
    for (int k = 0; k < TF_XPC; ++k) {
      const int i = ptid + k * TF_PROD;
      if (i >= TF_P * 8) continue;
      const int p = i >> 3, gq = i & 7;
      const int x = xb + TF_KC * c + 4 * gq;
      const int r = T.row0 + p;
      const bool ok = p < T.npen && x < PX;
      const float* src = ok ? in + (long long)(r % N2) * sy + (long long)(r / N2) * sz + x : in;
      cp_async16(sdst + tf_cell(p, gq), src, ok);
    }
  } else {
    const int Nax = P.N[AXIS];
#pragma unroll
    for (int b = 0; b < TF_BLK; ++b) {
      const int i = ptid + b * TF_PROD;
      if (i >= 256) continue;
      const int pg = i & 31, kq = i >> 5;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = T.lo + TF_KC * c + 4 * kq + r;
        const bool ok = row < Nax && T.x0 + 4 * pg < PX;
        const float* src = ok ? in + T.base0 + (long long)row * T.estride + 4 * pg : in;
        cp_async16(sdst + tf_cell(4 * pg + r, kq), src, ok);
      }
    }
  }
}

__device__ __forceinline__ float4 ld_shared4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a)
               : "memory");
  return v;
}

__device__ __forceinline__ void st_shared4(uint32_t d, float a, float b, float c, float e) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(d), "f"(a), "f"(b), "f"(c), "f"(e) : "memory");
}

// The in-place pass over this thread's cells of a landed stage: every value rounded to the
// nearest TF32 (the tensor cores would drop the low bits instead), y and z blocks transposed.
template <int AXIS>
__device__ __forceinline__ void tf_process(uint32_t sdst, int ptid) {
  if (AXIS == 0) {
#pragma unroll
    for (int k = 0; k < TF_XPC; ++k) {
      const int i = ptid + k * TF_PROD;
      if (i >= TF_P * 8) continue;
      const uint32_t a = sdst + tf_cell(i >> 3, i & 7);
      const float4 v = ld_shared4(a);
      st_shared4(a, tf32r(v.x), tf32r(v.y), tf32r(v.z), tf32r(v.w));
    }
  } else {
#pragma unroll
    for (int b = 0; b < TF_BLK; ++b) {
      const int i = ptid + b * TF_PROD;
      if (i >= 256) continue;
      const int pg = i & 31, kq = i >> 5;
      float4 v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = ld_shared4(sdst + tf_cell(4 * pg + r, kq));
      st_shared4(sdst + tf_cell(4 * pg, kq), tf32r(v[0].x), tf32r(v[1].x), tf32r(v[2].x), tf32r(v[3].x));
      st_shared4(sdst + tf_cell(4 * pg + 1, kq), tf32r(v[0].y), tf32r(v[1].y), tf32r(v[2].y), tf32r(v[3].y));
      st_shared4(sdst + tf_cell(4 * pg + 2, kq), tf32r(v[0].z), tf32r(v[1].z), tf32r(v[2].z), tf32r(v[3].z));
      st_shared4(sdst + tf_cell(4 * pg + 3, kq), tf32r(v[0].w), tf32r(v[1].w), tf32r(v[2].w), tf32r(v[3].w));
    }
  }
}

// ---- barriers ----------------------------------------------------------------------------
struct TfBars {
  uint64_t* full;       // [nst] TF_PROD arrivals + 1 (matrix copy, transaction bytes)
  uint64_t* empty;      // [nst] 1 (MMA commit): the stage has been read
  uint64_t* acc_full;   // [2]   1 (MMA commit): the tile's contraction is done
  uint64_t* acc_empty;  // [2]   TF_EPI arrivals: the accumulator has been drained
  uint64_t* done;       // 1     (MMA commit): every MMA of the CTA has completed
  uint64_t* land;       // [nst] x axis: 1 (the TMA issuer) + the tile's transaction bytes
  uint64_t* xready;     // [2]   TF_PROD arrivals: a tile's partial sums of output 256 are written
  uint64_t* xfree;      // [2]   TF_EPI arrivals: the epilogue has read them
};

// ---- the MMA thread (warp 15, lane 0): matrix copies ahead, MMAs as stages land -----------
template <int AXIS>
__device__ void tf_mma_thread(const TfPassParams& P, const TfGeom& g, unsigned char* stages, const TfBars& B,
                              uint32_t tmem, int nacc, int my_tiles, volatile int* abort) {
  // chunk sequence: tile i, chunk c; loader position (li, lc), consumer position (ci, cc)
  int li = 0, lc = 0, ci = 0, cc = 0, cstarted = 0;
  long long nl = 0, nc = 0;  // chunks loaded, consumed
  TfTile LT, CT;
  if (my_tiles > 0) {
    LT = tf_tile_of<AXIS>(P, blockIdx.x);
    CT = LT;
  }
  long long idle = 0;
  while (ci < my_tiles) {
    bool progress = false;
    // -- loader: the next matrix chunk once its stage has been released
    if (li < my_tiles && nl < nc + g.nst) {
      const int s = (int)(nl % g.nst);
      const long long u = nl / g.nst;
      if (u == 0 || bar_test(&B.empty[s], (uint32_t)((u - 1) & 1))) {
        const TfGeom tg = TfGeom::make(LT.Kn, AXIS);
        const uint32_t mbytes = (uint32_t)tg.mp * TF_KC * 4;
        bulk_load(stages + (size_t)s * g.stage + TF_TILE_BYTES,
                  reinterpret_cast<const unsigned char*>(P.A[LT.q]) + (size_t)lc * mbytes, mbytes, &B.full[s]);
        ++nl;
        progress = true;
        if (++lc == LT.Kp / TF_KC) {
          lc = 0;
          if (++li < my_tiles) LT = tf_tile_of<AXIS>(P, blockIdx.x + li * gridDim.x);
        }
      }
    }
    // -- consumer: a tile starts once its accumulator is free
    const int a = ci % nacc;
    if (!cstarted) {
      if (ci < nacc || bar_test(&B.acc_empty[a], (uint32_t)(((ci / nacc) - 1) & 1))) {
        cstarted = 1;
        progress = true;
      }
    }
    if (cstarted && nc < nl) {
      const int s = (int)(nc % g.nst);
      if (bar_test(&B.full[s], (uint32_t)((nc / g.nst) & 1))) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const TfGeom cg = TfGeom::make(CT.Kn, AXIS);
        const uint32_t acc = tmem + (uint32_t)(a * 256);
        const uint32_t st = smem_u32(stages + (size_t)s * g.stage);
        const uint32_t sm = st + TF_TILE_BYTES;
#pragma unroll
        for (int ks = 0; ks < TF_KC / 8; ++ks) {
          const uint32_t accum = (cc > 0 || ks > 0) ? 1u : 0u;
          if (AXIS == 0) {
            // D[m][p] += T[m][k] S[p][k]: A = matrix (K-major, blocks of 128 rows), B = tile
            // (K-major, N = 128): a k-step of 8 is two core matrices along K
            const uint64_t db = smem_desc_sw128(st + (uint32_t)ks * 32u);
            for (int mb = 0; mb < cg.mp / 128; ++mb) {
              const uint64_t da = smem_desc(sm + (uint32_t)mb * 16u * 1024u + (uint32_t)ks * 256u, 128, 1024);
              tf_mma(acc + mb * 128, da, db, tf_idesc(TF_P), accum);
            }
          } else {
            // D[p][k] += S[p][j] T[k][j]: A = tile (K-major, M = 128 pencils), B = matrix
            // (K-major, N = outputs in blocks of up to 256)
            const uint64_t da = smem_desc(st + (uint32_t)ks * 256u, 128, 1024);
            for (int n0 = 0; n0 < CT.Kn; n0 += 256) {
              const int nn = CT.Kn - n0 < 256 ? CT.Kn - n0 : 256;
              const uint64_t db = smem_desc(sm + (uint32_t)(n0 / 8) * 1024u + (uint32_t)ks * 256u, 128, 1024);
              tf_mma(acc + n0, da, db, tf_idesc(nn), accum);
            }
          }
        }
        mma_commit(&B.empty[s]);
        ++nc;
        progress = true;
        if (++cc == CT.Kp / TF_KC) {
          mma_commit(&B.acc_full[a]);
          cc = 0;
          cstarted = 0;
          if (++ci < my_tiles) CT = tf_tile_of<AXIS>(P, blockIdx.x + ci * gridDim.x);
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
  for (long long k = nc; k < nl; ++k) {
    const int s = (int)(k % g.nst);
    for (long long it = 0; it < UM_SPIN && !bar_test(&B.full[s], (uint32_t)((k / g.nst) & 1)); ++it) {
      if (*abort && it > 4096) break;  // a stage whose producers gave up never completes
      __nanosleep(64);
    }
  }
  if (nc > 0) {
    mma_commit(B.done);
    for (long long it = 0; it < UM_SPIN && !bar_test(B.done, 0u); ++it) __nanosleep(64);
  }
}

// ---- Green factor along one z line (z forward pass, mode 2) -------------------------------
// With (kx, ky) fixed the B0 / 2 mu0 denominator 2 mu0 (a0 + a1 + a2) + lam0 a_q is
// alpha cz + beta sz (each a_i a sum of monomials in the squared sines and cosines, linear in
// cz and sz); a monomial with a zero factor stays exactly zero, so null denominators stay
// exact zeros.
struct TfGreenLine {
  float alpha, beta, g;
  __device__ __forceinline__ float at(float sz, float cz) const {
    const float den = fmaf(alpha, cz, beta * sz);
    return den > 0.f ? __fdividef(g, den) : 0.f;
  }
};

__device__ __forceinline__ TfGreenLine tf_green_line(const TfPassParams& P, int q, int kx, int ky) {
  const float sx = P.S2[q][0][kx], cx = P.C2[q][0][kx];
  const float sy = P.S2[q][1][ky], cy = P.C2[q][1][ky];
  const float t = P.tetra ? 1.f : 0.f;
  const float c00 = P.hf[0] * sx * cy, c01 = t * P.hf[0] * cx * sy;
  const float c10 = P.hf[1] * cx * sy, c11 = t * P.hf[1] * sx * cy;
  const float c20 = t * P.hf[2] * sx * sy, c21 = P.hf[2] * cx * cy;
  const float aqc = q == 0 ? c00 : (q == 1 ? c10 : c20);
  const float aqs = q == 0 ? c01 : (q == 1 ? c11 : c21);
  TfGreenLine G;
  G.alpha = P.two_mu0 * (c00 + c10 + c20) + P.lam0 * aqc;
  G.beta = P.two_mu0 * (c01 + c11 + c21) + P.lam0 * aqs;
  G.g = -P.gscale[q];
  return G;
}

// ---- the epilogue (warps 0-7) --------------------------------------------------------------
// Warp w reads TMEM lanes 32 (w % 4) .. + 31 and takes half h = w / 4 of the accumulator's
// columns (x: of its M blocks).
// The Green factor's per-tile inputs, fetched by each epilogue warp before it waits for the
// accumulator (their latency hides behind the wait): the (kx, ky) line coefficients and, when a
// warp's half of the z outputs spans at most TF_ZCH chunks of 16, that half's sin^2 / cos^2
// factors, chunk j in register r[j] (lane i < 16: sin^2 of output 16 j + i; lane 16 + i: cos^2).
constexpr int TF_ZCH = 8;
struct TfZPre {
  TfGreenLine G;
  bool gl, reg;
  float r[TF_ZCH];
};

__device__ __forceinline__ TfZPre tf_z_prefetch(const TfPassParams& P, const TfTile& T, int warp, int lane) {
  TfZPre Z;
  const int q = T.q, p = (warp & 3) * 32 + lane, h = warp >> 2, half = T.Kn / 2;
  const int kx = T.x0 + p - P.flo[q][0], ky = T.other - P.flo[q][1];
  Z.gl = p < T.npen && kx >= 0 && kx < P.fL[q][0] && ky >= 0 && ky < P.fL[q][1];
  Z.G = tf_green_line(P, q, Z.gl ? kx : 0, Z.gl ? ky : 0);
  Z.reg = half <= 16 * TF_ZCH;
  const float* __restrict__ src = lane < 16 ? P.S2[q][2] : P.C2[q][2];
#pragma unroll
  for (int j = 0; j < TF_ZCH; ++j) {
    const int k = min(h * half + 16 * j + (lane & 15), T.L - 1);
    Z.r[j] = (Z.reg && 16 * j < half) ? __ldg(src + k) : 0.f;
  }
  return Z;
}

template <int AXIS>
__device__ __forceinline__ void tf_store_tile(const TfPassParams& P, const TfTile& T, uint32_t acc, int warp,
                                              int lane, const TfZPre& Z) {
  const int q = T.q, L = T.L, Kp = T.Kn, npen = T.npen;  // Kp: the outputs in TMEM
  float* __restrict__ out = P.out[q];
  const float sc = P.scale[q];
  const int gq = warp & 3, h = warp >> 2;
  const uint32_t lane_base = (uint32_t)(gq * 32) << 16;
  if (AXIS == 0) {
    // lanes are outputs: M index m <-> node x = xb + m; a warp writes 32 consecutive nodes of
    // one row per store
    const float* __restrict__ bh = P.base[q];
    const float* __restrict__ bl = P.base_lo[q];
    float* __restrict__ ol = P.out_lo[q];
    const int mp = (Kp + 127) / 128 * 128, xb = T.lo & ~3;
    const int N2 = P.N[1];
    const long long sy = P.stride[1], wrap = P.stride[2] - (long long)(N2 - 1) * P.stride[1];
    for (int mb = h; mb < mp / 128; mb += 2) {
      const int x = xb + mb * 128 + gq * 32 + lane;
      const bool ok = x >= T.lo && x < T.lo + L;
      // 16 rows per round, the loop rolled (a compact body: the epilogue shares the
      // instruction cache with the producers and the MMA thread)
      const bool acc_mode = P.mode == 1 && bh != nullptr;
      const int wr = (int)wrap, syi = (int)sy;
#pragma unroll 1
      for (int p0 = 0; p0 < npen; p0 += 16) {
        float v[16];
        tmem_ld16(acc + lane_base + (uint32_t)(mb * 128 + p0), v);  // warp-collective
        if (!ok) continue;
        // row r = row0 + p0 + u of the grid's (y, z) rows: its offset advances by sy, or
        // wraps to the next z plane
        int y = (T.row0 + p0) % N2;
        int row = y * syi + ((T.row0 + p0) / N2) * (int)P.stride[2];  // within one component array
        int at[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          at[u] = row + x;
          row += (++y == N2) ? wr : syi;
          if (y == N2) y = 0;
        }
        if (!acc_mode) {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (p0 + u < npen) out[at[u]] = sc * v[u];
        } else {
          // the base values of the 16 rows are loaded before the first sum (loads in flight together)
          float a[16], b[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const bool live = p0 + u < npen;
            a[u] = live ? bh[at[u]] : 0.f;
            b[u] = (live && ol) ? bl[at[u]] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (p0 + u >= npen) continue;
            const int o = at[u];
            const float val = sc * v[u];
            if (ol == nullptr) {
              out[o] = a[u] + val;
            } else {  // (hi, lo) = (bh, bl) + val with an error-free sum of the high parts
              const float s1 = a[u] + val;
              const float bs = s1 - a[u];
              const float er = (a[u] - (s1 - bs)) + (val - bs);
              const float tt = b[u] + er;
              const float hsum = s1 + tt;
              out[o] = hsum;
              ol[o] = tt - (hsum - s1);
            }
          }
        }
      }
    }
  } else {
    // lanes are pencils (consecutive in memory): one coalesced store per output
    const int p = gq * 32 + lane;
    const bool live = p < npen;
    const long long rowbase = T.base0 + p + (long long)T.lo * T.estride;
    const bool green = AXIS == 2 && P.mode == 2;
    const int half = Kp / 2;  // a multiple of 16
    if (green && Z.reg) {
      // the z factors come from the prefetched registers, one shuffle per factor.  The chunk
      // loop stays rolled: a compact body, since the epilogue shares the instruction cache
      // with the producers and the MMA thread
      const float gs = Z.gl ? Z.G.g * sc : 0.f;  // the scale folded into the factor's numerator
      const float al = Z.G.alpha, be = Z.G.beta;
      const long long es = T.estride;
      const int nch = half / 16;
      float* o = out + rowbase + (long long)(h * half) * es;
#pragma unroll 1
      for (int j = 0; j < nch; ++j) {
        const int kb = h * half + 16 * j;
        const float zr = Z.r[j];
        float v[16];
        tmem_ld16(acc + lane_base + (uint32_t)kb, v);  // warp-collective: every lane takes part
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float zs = __shfl_sync(0xffffffffu, zr, i);
          const float zc = __shfl_sync(0xffffffffu, zr, 16 + i);
          const float den = fmaf(al, zc, be * zs);
          const float f = den > 0.f ? __fdividef(gs, den) : 0.f;
          if (live && kb + i < L) o[(long long)i * es] = v[i] * f;
        }
        o += 16 * es;
      }
      return;
    }
    const TfGreenLine& G = Z.G;
    const bool gl = Z.gl;
    const float* __restrict__ Sz = P.S2[q][2];
    const float* __restrict__ Cz = P.C2[q][2];
    for (int c0 = h * half; c0 < (h + 1) * half; c0 += 16) {
      float zs[16], zc[16];
      if (green) {  // the z factors of these 16 outputs, loaded before the TMEM read
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = min(c0 + i, L - 1);
          zs[i] = __ldg(Sz + k);
          zc[i] = __ldg(Cz + k);
        }
      }
      float v[16];
      tmem_ld16(acc + lane_base + (uint32_t)c0, v);  // warp-collective: every lane takes part
      if (!live) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = c0 + i;
        if (k >= L) continue;
        float val = sc * v[i];
        if (green) val = gl ? val * G.at(zs[i], zc[i]) : 0.f;
        out[rowbase + (long long)k * T.estride] = val;
      }
    }
  }
}

template <int AXIS>
__global__ void __launch_bounds__(TF_THREADS, 1) k_pass_tf32(const __grid_constant__ TfPassParams P, int maxKn,
                                                              int xtra) {
  if (P.stop && *P.stop) return;  // before any TMEM allocation or barrier
  extern __shared__ __align__(1024) unsigned char smem[];
  const TfGeom g = TfGeom::make(maxKn, AXIS, xtra);
  // fixed region (2 KB): barriers, TMEM slot, abort flag; the stages follow
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  TfBars B;
  B.full = bars;
  B.empty = bars + TF_MAXST;
  B.acc_full = bars + 2 * TF_MAXST;
  B.acc_empty = bars + 2 * TF_MAXST + 2;
  B.done = bars + 2 * TF_MAXST + 4;
  B.land = bars + 2 * TF_MAXST + 5;
  B.xready = bars + 3 * TF_MAXST + 5;
  B.xfree = bars + 3 * TF_MAXST + 7;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * TF_MAXST + 9);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  unsigned char* stages = smem + 2048;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the x tiles use the 128-byte swizzle, whose pattern the MMA descriptor takes from 1024-byte
  // aligned stages (every stage size is a multiple of 1024): refuse a misaligned window
  if (AXIS == 0 && (smem_u32(stages) & 1023u)) {
    if (tid == 0) atomicExch(P.err, 1);
    return;
  }
  const int ntiles = tf_total_tiles<AXIS>(P);
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nacc = 2 * g.acc_cols <= TF_TMEM_COLS ? 2 : 1;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(TF_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int s = 0; s < TF_MAXST; ++s) {
      bar_init(&B.full[s], TF_PROD + 1);
      bar_init(&B.empty[s], 1);
      bar_init(&B.land[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&B.acc_full[i], 1);
      bar_init(&B.acc_empty[i], TF_EPI);
      bar_init(&B.xready[i], TF_PROD);
      bar_init(&B.xfree[i], TF_EPI);
    }
    bar_init(B.done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp >= TF_EPI / 32 && warp < (TF_EPI + TF_PROD) / 32) {
    // ---- producers: the tile part of every stage; up to `depth` stages of copies in flight,
    // the oldest processed and handed to the MMA thread as soon as it has landed ----
    const int ptid = tid - TF_EPI;
    if (AXIS == 0 || g.raw) {
      // one thread issues a TMA box per stage.  x: 32 x values of 128 consecutive rows, written in
      // the 128-byte-swizzled K-major layout; once it has landed every producer rounds its share of
      // the 16 KB to the nearest TF32 in place.  y, z: 32 rows along the axis of 128 consecutive
      // pencils, into the stage's raw part; every producer transposes its 4 x 4 blocks from there
      // into the K-major tile, rounded
      const int depth = g.nst - 1 < 3 ? g.nst - 1 : 3;
      long long seq = 0, done = 0;
      int ti = 0, c = 0;
      TfTile T;
      if (my_tiles > 0) T = tf_tile_of<AXIS>(P, blockIdx.x);
      // output 256 of a 257-output transform (y, z): each producer keeps the partial dot products
      // of its two 4 x 4 blocks (row group kq, pencils 4 pg ..) over the tile's chunks and stores
      // them, per row group, in one of two slot sets; the epilogue adds the eight row groups in order
      TfTile PT;  // the tile being processed, its chunk and its rank among the tiles with xt
      int pc = 0, pti = 0, pxi = 0;
      if (my_tiles > 0) PT = T;
      float xacc[TF_BLK][4];
#pragma unroll
      for (int b = 0; b < TF_BLK; ++b)
#pragma unroll
        for (int j = 0; j < 4; ++j) xacc[b][j] = 0.f;
      float* const xpart = reinterpret_cast<float*>(stages + g.xoff());
      auto process = [&](long long k) {
        const int s = (int)(k % g.nst);
        if (!bar_wait(&B.land[s], (uint32_t)((k / g.nst) & 1), abort)) return false;
        const uint32_t base = smem_u32(stages + (size_t)s * g.stage);
        if (AXIS == 0) {
#pragma unroll
          for (int j = 0; j < TF_XPC; ++j) {
            const int i = ptid + j * TF_PROD;
            if (i >= TF_P * 8) continue;
            const float4 v = ld_shared4(base + (uint32_t)i * 16u);
            st_shared4(base + (uint32_t)i * 16u, tf32r(v.x), tf32r(v.y), tf32r(v.z), tf32r(v.w));
          }
        } else {
          const uint32_t raw = base + g.raw_off();
#pragma unroll
          for (int b = 0; b < TF_BLK; ++b) {
            const int i = ptid + b * TF_PROD;
            if (i >= 256) continue;
            const int pg = i & 31, kq = i >> 5;
            float4 v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) v[r] = ld_shared4(raw + (uint32_t)((4 * kq + r) * TF_P + 4 * pg) * 4u);
            if (AXIS != 0 && PT.xt) {  // FP32 tile values, FP32 matrix row
              const float* xr = P.xrow[PT.q] + TF_KC * pc + 4 * kq;
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const float w = __ldg(xr + r);
                xacc[b][0] = fmaf(w, v[r].x, xacc[b][0]);
                xacc[b][1] = fmaf(w, v[r].y, xacc[b][1]);
                xacc[b][2] = fmaf(w, v[r].z, xacc[b][2]);
                xacc[b][3] = fmaf(w, v[r].w, xacc[b][3]);
              }
            }
            st_shared4(base + tf_cell(4 * pg, kq), tf32r(v[0].x), tf32r(v[1].x), tf32r(v[2].x), tf32r(v[3].x));
            st_shared4(base + tf_cell(4 * pg + 1, kq), tf32r(v[0].y), tf32r(v[1].y), tf32r(v[2].y), tf32r(v[3].y));
            st_shared4(base + tf_cell(4 * pg + 2, kq), tf32r(v[0].z), tf32r(v[1].z), tf32r(v[2].z), tf32r(v[3].z));
            st_shared4(base + tf_cell(4 * pg + 3, kq), tf32r(v[0].w), tf32r(v[1].w), tf32r(v[2].w), tf32r(v[3].w));
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        bar_arrive(&B.full[s]);
        if (AXIS != 0 && ++pc == PT.Kp / TF_KC) {  // the tile's last chunk
          if (PT.xt) {
            const int par = pxi & 1;
            // the slot set was last read for the tile with xt two before this one
            if (pxi >= 2 && !bar_wait(&B.xfree[par], (uint32_t)(((pxi >> 1) - 1) & 1), abort)) return false;
#pragma unroll
            for (int b = 0; b < TF_BLK; ++b) {
              const int i = ptid + b * TF_PROD;
              if (i < 256) {
                const int pg = i & 31, kq = i >> 5;
#pragma unroll
                for (int j = 0; j < 4; ++j) xpart[(par * 8 + kq) * TF_P + 4 * pg + j] = xacc[b][j];
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) xacc[b][j] = 0.f;
            }
            bar_arrive(&B.xready[par]);
            ++pxi;
          }
          pc = 0;
          if (++pti < my_tiles) PT = tf_tile_of<AXIS>(P, blockIdx.x + pti * gridDim.x);
        }
        return true;
      };
      bool live = true;
      while (ti < my_tiles && live) {
        const int s = (int)(seq % g.nst);
        const long long u = seq / g.nst;
        if (ptid == 0) {
          if (u > 0 && !bar_wait(&B.empty[s], (uint32_t)((u - 1) & 1), abort)) break;
          expect_tx(&B.land[s], TF_TILE_BYTES);
          const uint32_t dst = smem_u32(stages + (size_t)s * g.stage);
          if (AXIS == 0)
            tma_load_2d(dst, &P.tmap[T.q], (T.lo & ~3) + TF_KC * c, T.row0, &B.land[s]);
          else if (AXIS == 1)
            tma_load_3d(dst + g.raw_off(), &P.tmap[T.q], T.x0, T.lo + TF_KC * c, T.other, &B.land[s]);
          else
            tma_load_3d(dst + g.raw_off(), &P.tmap[T.q], T.x0, T.other, T.lo + TF_KC * c, &B.land[s]);
        }
        ++seq;
        if (++c == T.Kp / TF_KC) {
          c = 0;
          if (++ti < my_tiles) T = tf_tile_of<AXIS>(P, blockIdx.x + ti * gridDim.x);
        }
        if (seq - done == depth) live = process(done++);
      }
      // the stages still in flight (thread 0 may have issued one more than the others counted
      // after an abort: every thread drains what it counted, thread 0 its own count)
      while (done < seq && live) live = process(done++);
    } else {
    const int depth = g.nst - 1 < 3 ? g.nst - 1 : 3;
    long long seq = 0, done = 0;  // stages issued, stages handed over
    int ti = 0, c = 0;
    TfTile T;
    if (my_tiles > 0) T = tf_tile_of<AXIS>(P, blockIdx.x);
    while (ti < my_tiles) {
      const int s = (int)(seq % g.nst);
      const long long u = seq / g.nst;
      if (u > 0 && !bar_wait(&B.empty[s], (uint32_t)((u - 1) & 1), abort)) break;
      tf_issue<AXIS>(P, T, c, ptid, smem_u32(stages + (size_t)s * g.stage));
      cp_async_commit();
      ++seq;
      if (++c == T.Kp / TF_KC) {
        c = 0;
        if (++ti < my_tiles) T = tf_tile_of<AXIS>(P, blockIdx.x + ti * gridDim.x);
      }
      if (seq - done == depth) {
        cp_async_wait(depth - 1);
        tf_process<AXIS>(smem_u32(stages + (size_t)(done % g.nst) * g.stage), ptid);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        bar_arrive(&B.full[(int)(done % g.nst)]);
        ++done;
      }
    }
    // the stages still in flight (all of them after an abort, whose copies must land before exit)
    cp_async_wait(0);
    for (; done < seq; ++done) {
      tf_process<AXIS>(smem_u32(stages + (size_t)(done % g.nst) * g.stage), ptid);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      bar_arrive(&B.full[(int)(done % g.nst)]);
    }
    }
  } else if (warp == (TF_EPI + TF_PROD) / 32) {
    // ---- warp 15: lane 0 copies the matrix chunks and issues the MMAs ----
    if (lane == 0) tf_mma_thread<AXIS>(P, g, stages, B, tmem, nacc, my_tiles, abort);
    __syncwarp();
  } else {
    // ---- epilogue warps 0-7 ----
    uint32_t acc_uses[2] = {0u, 0u};
    int xi = 0;  // rank of the tile among those whose output 256 the producers contract
    const float* const xpart = reinterpret_cast<const float*>(stages + g.xoff());
    for (int i = 0; i < my_tiles; ++i) {
      const int a = i % nacc;
      const uint32_t acc = tmem + (uint32_t)(a * 256);
      const TfTile T = tf_tile_of<AXIS>(P, blockIdx.x + i * gridDim.x);
      TfZPre Z;
      Z.gl = Z.reg = false;
      Z.G.alpha = Z.G.beta = Z.G.g = 0.f;
      if (AXIS == 2 && P.mode == 2) Z = tf_z_prefetch(P, T, warp, lane);
      if (!bar_wait(&B.acc_full[a], acc_uses[a] & 1, abort)) break;
      ++acc_uses[a];
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      tf_store_tile<AXIS>(P, T, acc, warp, lane, Z);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      bar_arrive(&B.acc_empty[a]);
      if (AXIS != 0 && T.xt) {  // output 256: the producers' partial sums, row groups in order
        const int par = xi & 1;
        if (!bar_wait(&B.xready[par], (uint32_t)((xi >> 1) & 1), abort)) break;
        const int p = (warp & 3) * 32 + lane;
        if ((warp >> 2) == 0 && p < T.npen && 256 < T.L) {
          float sum = 0.f;
#pragma unroll
          for (int kq = 0; kq < 8; ++kq) sum += xpart[(par * 8 + kq) * TF_P + p];
          float val = P.scale[T.q] * sum;
          if (AXIS == 2 && P.mode == 2) {  // the Green factor at frequency 256 of this (kx, ky) line
            const float gs = Z.gl ? Z.G.g * P.scale[T.q] : 0.f;
            const float den = fmaf(Z.G.alpha, __ldg(P.C2[T.q][2] + 256), Z.G.beta * __ldg(P.S2[T.q][2] + 256));
            val = sum * (den > 0.f ? __fdividef(gs, den) : 0.f);
          }
          P.out[T.q][T.base0 + p + (long long)(T.lo + 256) * T.estride] = val;
        }
        bar_arrive(&B.xfree[par]);
        ++xi;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(P.err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TF_TMEM_COLS));
}

template <int AXIS>
static cudaError_t launch_tf32_one(const TfPassParams& P, int maxKn, int xtra, cudaStream_t s) {
  const size_t smem = TfGeom::make(maxKn, AXIS, xtra).smem();
  auto kern = k_pass_tf32<AXIS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one persistent CTA per SM (each holds all 512 TMEM columns)
  kern<<<dim3((unsigned)(sms > 0 ? sms : 152)), TF_THREADS, smem, s>>>(P, maxKn, xtra);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library links the
// runtime only)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// x axis: component q's input as {row pitch (x), N2 * N3 rows}, boxes of 32 x 128 with the
// 128-byte swizzle; coordinates past the extents read zeros
// y, z axes: component q's input as {row pitch, N2, N3}, boxes of 128 x values by 32 rows along
// the pass axis, no swizzle (the rows land one after the other in the stage's raw part)
static cudaError_t encode_maps(TfPassParams& P) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  for (int q = 0; q < 3; ++q) {
    CUresult r;
    if (P.axis == 0) {
      const cuuint64_t dims[2] = {(cuuint64_t)P.stride[1], (cuuint64_t)P.N[1] * (cuuint64_t)P.N[2]};
      const cuuint64_t strides[1] = {(cuuint64_t)P.stride[1] * sizeof(float)};
      const cuuint32_t box[2] = {(cuuint32_t)TF_KC, (cuuint32_t)TF_P};
      const cuuint32_t estr[2] = {1, 1};
      r = enc(&P.tmap[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(P.in[q]), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      const cuuint64_t dims[3] = {(cuuint64_t)P.stride[1], (cuuint64_t)P.N[1], (cuuint64_t)P.N[2]};
      const cuuint64_t strides[2] = {(cuuint64_t)P.stride[1] * sizeof(float), (cuuint64_t)P.stride[2] * sizeof(float)};
      const cuuint32_t box[3] = {(cuuint32_t)TF_P, P.axis == 1 ? (cuuint32_t)TF_KC : 1u, P.axis == 2 ? (cuuint32_t)TF_KC : 1u};
      const cuuint32_t estr[3] = {1, 1, 1};
      r = enc(&P.tmap[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(P.in[q]), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_pass_tf32(const TfPassParams& P0, cudaStream_t s) {
  TfPassParams P = P0;
  {
    const cudaError_t e = encode_maps(P);
    if (e != cudaSuccess) return e;
  }
  int maxKn = 0, xtra = 0;
  for (int q = 0; q < 3; ++q) {
    // output 256 in the producers: y, z only, 257 outputs, 256 of them on the tensor cores
    if (P.xrow[q] && (P.axis == 0 || P.Kn[q] != 256 || P.L[q] != 257)) return cudaErrorInvalidValue;
    xtra |= P.xrow[q] != nullptr;
    if (!P.xrow[q] && P.Kn[q] != P.Kp[q]) return cudaErrorInvalidValue;
    maxKn = maxKn > P.Kn[q] ? maxKn : P.Kn[q];
  }
  for (int q = 0; q < 3; ++q)
    if (!pass_tf32_fits(P.Kn[q], P.axis, xtra)) return cudaErrorInvalidValue;
  if (xtra && !TfGeom::make(maxKn, P.axis, 1).raw) return cudaErrorInvalidValue;  // TMA producers only
  if (P.mode == 1 && P.axis != 0) return cudaErrorInvalidValue;
  if (P.mode == 2 && P.axis != 2) return cudaErrorInvalidValue;
  if (P.axis == 0) return launch_tf32_one<0>(P, maxKn, xtra, s);
  if (P.axis == 1) return launch_tf32_one<1>(P, maxKn, xtra, s);
  return launch_tf32_one<2>(P, maxKn, xtra, s);
}

bool pass_tf32_fits(int Kn, int axis, int xtra) {
  if (Kn < TF_KC || Kn % TF_KC != 0) return false;
  const TfGeom g = TfGeom::make(Kn, axis, xtra);
  // the accumulator fits TMEM (x: Mp / 128 blocks of 128 columns; y, z: Kn columns) and the
  // ring has at least three stages
  return g.acc_cols <= TF_TMEM_COLS && g.nst >= 3 && g.smem() <= (size_t)kMaxDynSmem;
}

int pass_tf32_rows(int Kp, int axis) { return TfGeom::make(Kp, axis).mp; }

}  // namespace fftm
