// C ABI of the fftm library (include/fftm.h): problem setup and the solve
// loop of Algorithm 1 (Sec. 2.4) on one GPU and one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <math_constants.h>

#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/fftm.h"
#include "fftm_internal.cuh"

using namespace fftm;

static thread_local std::string g_last_error;

static int set_err(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return set_err(FFTM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

// a device allocation: FFTM_E_NOMEM when the device or the caller's workspace has no room
#define DEVALLOC(call)                                                                            \
  do {                                                                                            \
    if ((call) != cudaSuccess) {                                                                  \
      cudaGetLastError();                                                                         \
      return set_err(FFTM_E_NOMEM, std::string("device allocation failed: ") + #call);            \
    }                                                                                             \
  } while (0)

struct fftm_ctx {
  int device;
  cudaStream_t stream;
};

namespace {

const double kPi = 3.14159265358979323846;

// BC on a face -> symmetry of u^f_q (Sec. 2.2): +1 symmetric (Neumann), -1 anti-symmetric (Dirichlet).
int face_sym(int bc) { return bc == FFTM_BC_NEUMANN ? 1 : -1; }

// Pair of face symmetries -> transform kind (Table 1).
int kind_of(int left, int right, bool periodic) {
  if (periodic) return K_DFT;
  if (left > 0 && right > 0) return K_DCT1;
  if (left > 0 && right < 0) return K_DCT3;
  if (left < 0 && right < 0) return K_DST1;
  return K_DST3;
}

// Node range [lo, lo + L) of a kind (Table 1 index j; the rest is dismissed, Sec. 2.7.2).
void kind_range(int kind, int n, int* lo, int* L) {
  switch (kind) {
    case K_DFT: *lo = 0; *L = n; break;
    case K_DCT1: *lo = 0; *L = n + 1; break;
    case K_DCT3: *lo = 0; *L = n; break;
    case K_DST1: *lo = 1; *L = n - 1; break;
    default: *lo = 1; *L = n; break;
  }
}

// Fundamental frequency of index k (Table 1) and whether it is exactly 0 or pi.
double kind_xi(int kind, int n, int k, bool* zero, bool* pi) {
  *zero = false;
  *pi = false;
  switch (kind) {
    case K_DFT: *zero = (k == 0); *pi = (2 * k == n); return 2.0 * kPi * k / n;
    case K_DCT1: *zero = (k == 0); *pi = (k == n); return kPi * k / n;
    case K_DST1: return kPi * (k + 1) / n;
    default: return kPi * (k + 0.5) / n;
  }
}

bool factor_radices(int M, std::vector<int>* rad) {
  rad->clear();
  int m = M;
  while (m % 3 == 0) { rad->push_back(3); m /= 3; }
  while (m % 8 == 0) { rad->push_back(8); m /= 8; }
  while (m % 4 == 0) { rad->push_back(4); m /= 4; }
  while (m % 2 == 0) { rad->push_back(2); m /= 2; }
  return m == 1 && (int)rad->size() <= MAX_STAGES;
}

struct HostPlan {
  int kind, n, lo, L, M;
  std::vector<int> radix;
  std::vector<int16_t> perm;
  std::vector<double> tw;  // interleaved re, im
  std::vector<double> qw;
};

HostPlan make_plan(int kind, int n) {
  HostPlan p;
  p.kind = kind;
  p.n = n;
  kind_range(kind, n, &p.lo, &p.L);
  p.M = (kind == K_DFT) ? n : 2 * n;
  factor_radices(p.M, &p.radix);
  const int S = (int)p.radix.size();
  std::vector<int> Lw(S + 1, 1);  // Lw[s] = R_0 ... R_{s-1}
  for (int s = 0; s < S; ++s) Lw[s + 1] = Lw[s] * p.radix[s];
  p.perm.resize(p.M);
  for (int j = 0; j < p.M; ++j) {
    int rem = j, pos = 0;
    for (int s = S - 1; s >= 0; --s) {
      const int r = rem % p.radix[s];
      rem /= p.radix[s];
      pos += r * Lw[s];
    }
    p.perm[j] = (int16_t)pos;
  }
  p.tw.resize(2 * p.M);
  for (int t = 0; t < p.M; ++t) {
    const double a = -2.0 * kPi * t / p.M;
    p.tw[2 * t] = std::cos(a);
    p.tw[2 * t + 1] = std::sin(a);
  }
  p.qw.resize(2 * (n + 1));
  for (int j = 0; j <= n; ++j) {
    const double a = kPi * j / (2.0 * n);
    p.qw[2 * j] = std::cos(a);
    p.qw[2 * j + 1] = std::sin(a);
  }
  return p;
}

// Rotation of a unit quaternion (w, v): R = (w^2 - v.v) I + 2 v v^T + 2 w [v]_x.
void quat_rot(const double q[4], double R[3][3]) {
  double nrm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / nrm, v[3] = {q[1] / nrm, q[2] / nrm, q[3] / nrm};
  const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double X[3][3] = {{0, -v[2], v[1]}, {v[2], 0, -v[0]}, {-v[1], v[0], 0}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = (i == j ? w * w - vv : 0.0) + 2.0 * v[i] * v[j] + 2.0 * w * X[i][j];
}

// Mandel 6x6 of the cubic stiffness (C11, C12, C44) rotated by R (crystal -> sample).
void cubic_mandel(double C11, double C12, double C44, const double R[3][3], double Cm[6][6]) {
  double C0[3][3][3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          double v = 0.0;
          if (a == b && c == d) v += (a == c) ? C11 : C12;
          if (a != b && ((a == c && b == d) || (a == d && b == c))) v += C44;
          C0[a][b][c][d] = v;
        }
  static const int I2[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      const int i = I2[I][0], j = I2[I][1], k = I2[J][0], l = I2[J][1];
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d)
              if (C0[a][b][c][d] != 0.0) s += R[i][a] * R[j][b] * R[k][c] * R[l][d] * C0[a][b][c][d];
      const double f = (I >= 3 ? std::sqrt(2.0) : 1.0) * (J >= 3 ? std::sqrt(2.0) : 1.0);
      Cm[I][J] = f * s;
    }
}

// Dense forward matrix of a Table 1 transform over its node range (rows k,
// columns j - lo): periodic axes in halfcomplex order (real part of frequency k
// in row k, imaginary part in row n - k).
void dense_forward(int kind, int n, std::vector<double>* M, int* Lout) {
  int lo, L;
  kind_range(kind, n, &lo, &L);
  *Lout = L;
  M->assign((size_t)L * L, 0.0);
  for (int k = 0; k < L; ++k)
    for (int c = 0; c < L; ++c) {
      const int j = lo + c;
      double v = 0.0;
      switch (kind) {
        case K_DFT:
          if (2 * k <= n) v = std::cos(2.0 * kPi * j * k / n);
          else v = -std::sin(2.0 * kPi * j * (n - k) / n);
          break;
        case K_DCT1: v = (2.0 - (j == 0) - (j == n)) * std::cos(kPi * j * k / n); break;
        case K_DCT3: v = (2.0 - (j == 0)) * std::cos(kPi * j * (k + 0.5) / n); break;
        case K_DST1: v = 2.0 * std::sin(kPi * j * (k + 1.0) / n); break;
        default: v = (2.0 - (j == n)) * std::sin(kPi * j * (k + 0.5) / n); break;
      }
      (*M)[(size_t)k * L + c] = v;
    }
}

// Its exact inverse (rows j - lo, columns k): DCT-I/(2n), DCT-II/(2n),
// DST-I/(2n), DST-II/(2n), and the halfcomplex-to-real DFT divided by n.
void dense_inverse(int kind, int n, std::vector<double>* M) {
  int lo, L;
  kind_range(kind, n, &lo, &L);
  M->assign((size_t)L * L, 0.0);
  for (int r = 0; r < L; ++r)
    for (int k = 0; k < L; ++k) {
      const int j = lo + r;
      double v = 0.0;
      switch (kind) {
        case K_DFT:
          if (2 * k <= n) v = ((k == 0 || 2 * k == n) ? 1.0 : 2.0) * std::cos(2.0 * kPi * j * k / n) / n;
          else v = -2.0 * std::sin(2.0 * kPi * j * (n - k) / n) / n;
          break;
        case K_DCT1: v = (2.0 - (k == 0) - (k == n)) * std::cos(kPi * j * k / n) / (2.0 * n); break;
        case K_DCT3: v = std::cos(kPi * j * (k + 0.5) / n) / n; break;
        case K_DST1: v = std::sin(kPi * j * (k + 1.0) / n) / n; break;
        default: v = std::sin(kPi * j * (k + 0.5) / n) / n; break;
      }
      (*M)[(size_t)r * L + k] = v;
    }
}

// Round to TF32 (10 explicit significand bits; nearest, ties to even) from FP64 through FP32,
// so that the tensor cores read the matrix entries exactly.
float to_tf32(double d) {
  const float f = (float)d;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0xFFFu + ((b >> 13) & 1u);
  b &= ~0x1FFFu;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// Round to BF16 (nearest, ties to even) from FP64 through FP32.
uint16_t to_bf16(double d) {
  const float f = (float)d;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}

}  // namespace

struct fftm_problem {
  fftm_ctx* ctx = nullptr;
  fftm_problem_desc desc;
  std::vector<fftm_material> mats;
  int prec = FFTM_FP64;
  int tetra = 0;
  int n[3], N[3], periodic[3];
  double h[3];
  long long PX, sy, sz, comp_stride, nvox;
  int kind[3][3], lo[3][3], hi[3][3], sgn[3][3][2];
  HostPlan plans[3][3];  // [q][axis]
  fftm_load load;
  long long launches = 0;

  // device memory (type-erased; element size esz)
  size_t esz = 8;
  void* fields = nullptr;  // 11 sets x 3 comps
  void* Dbuf = nullptr;    // 3 comps, allocated on first FFTM_OP_RESIDUAL
  void* tables = nullptr;  // plans + green tables
  uint16_t* phase = nullptr;
  int* law_id = nullptr;
  void* law_c = nullptr;
  void* law_m = nullptr;  // elastic phases: the 6x6 Mandel stiffness in (2 x 2)-pair order, 36 per phase
  double* partial = nullptr;
  size_t partial_len = 0;
  double* dscal = nullptr;  // [0..1] norms, [2..9] anderson coef, [16..] stats
  int* dint = nullptr;      // accepted flags per iteration
  int dint_len = 0;
  double* hpin = nullptr;   // pinned host scalars
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* vs = nullptr;       // voxel-point stresses of the solver (NPP x NC x nvox)
  void* vs_test = nullptr;  // with tau, for FFTM_OP_RESIDUAL (allocated on first use)
  int sym = 1;              // every law gives a symmetric P
  void* state = nullptr;    // committed J2 state [r][7][voxel]: elastic strain e_n, p_n (only if a phase is J2)
  void* un = nullptr;       // u^f at the last commit: 3 comps (FP64) or 3 high + 3 low (FP32)
  fftm_load load_n;         // the load at the last commit
  double mixed_A[3][3];     // A at the end of the last normal-mixed step
  int mixed_prev = 0;       // that step's mask (0: none since creation or reset)
  void* Dn = nullptr;       // residual D at the last commit (3 comps)
  int committed = 0;        // a load step has been committed since creation or reset
  int nst = 0;              // state components per voxel point (7 J2 and logarithmic J2, 10 crystal plasticity, 0 none)
  int slaw = 0;             // 1 J2, 2 crystal plasticity, 4 logarithmic J2, 0 none
  int c0 = 0;               // the C0 Green operator (three components coupled per frequency)
  void* tface[3][2] = {};   // non-uniform tractions per face (fftm_set_face_traction), or null
  void* tface_n[3][2] = {}; // the fields at the last commit (J2's incremental residual)
  char* arena = nullptr;    // caller-provided device workspace (fftm_problem_create_in), or null
  size_t arena_size = 0, arena_used = 0;
  void* ustar = nullptr;    // u* as a node field (fftm_set_load_field), 3 components, or null
  void* ustar_n = nullptr;  // that field at the last commit (J2's incremental residual)
  void* c0tab = nullptr;    // its sin / cos tables per axis over the node positions
  void* state_next = nullptr;  // the state committed by the last converged step, swapped in when
  int commit_pending = 0;      // the next step starts (readouts until then see the step's own state)
  int inc_ok = 0;           // incremental residual after a commit (J2 with linear small-strain laws)
  // tensor-core transforms (FFTM_FP32_TC): BF16 matrices, Kp x Kp per component and axis
  int tc = 0;
  int tf = 0;  // FFTM_FP32_TF32: FP32 matrices, TF32 contractions (same offsets tables)
  void* tcmat = nullptr;
  int* tc_err = nullptr;  // timeout flag of the tensor-core passes
  size_t off_tcf[3][3], off_tci[3][3];
  int tcKp[3][3];
  int tcKn[3][3];                        // TF32: outputs on the tensor cores (tcKp, or 256)
  size_t off_tcxf[3][3], off_tcxi[3][3];  // TF32 y, z with 257 outputs: output 256's row
  int tcx[3][3];
  // device table offsets (bytes) inside `tables`
  size_t off_perm[3][3], off_tw[3][3], off_qw[3][3], off_S2[3][3], off_C2[3][3];
  int maxM[3], maxL[3];
  int cur = 0;  // ring slot holding the current u^f
  int res_passes = 0;     // requested residual form: 0 tuned, 1 one pass, 2 two passes
  int res_two_pass = -1;  // resolved form (-1: not yet)
  int res_tile = 0;       // requested one-pass tile height: 0 tuned, 8 or 16
  int res_fy = 8;         // resolved tile height
  // per-kernel timing (fftm_set_profiling)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_free;
  struct Pending { int cat, a, b, m, post; };
  std::vector<Pending> pending;
  int prof_m = -1, prof_post = 0;  // iteration tag of the launches being enqueued (device loop)
  // device-decided load steps (every load without a normal-mixed part): the convergence test
  // runs on the device and the host waits once per chunk of iterations
  int dev_loop = 1;                // FFTM_OPT_DEVICE_LOOP
  int graph = 0;                   // FFTM_OPT_CUDA_GRAPH: device-decided steps replay captured iterations
  int last_iters = -1;             // iterations of the previous device-decided step (chunk sizing)
  int* dctl = nullptr;             // control block of k_check: stop, next iteration, last checked
  double* derr = nullptr;          // per-iteration errors of the step (device)
  int derr_len = 0;
  const int* stop = nullptr;       // dctl while a device-decided step is being enqueued, else null
  double prof_ms[FFTM_KCAT_COUNT] = {0, 0, 0, 0, 0, 0};
  long long prof_cnt[FFTM_KCAT_COUNT] = {0, 0, 0, 0, 0, 0};
};

namespace {

// Field sets (3 component arrays each).  u^f lives in a ring of NSLOT slots so
// that the last Anderson couples (u^k, D^k) stay in place without copies:
// iteration m reads u^m from slot (cur0 + m) % NSLOT, writes D^m to the D slot
// of the same index and u^{m+1} to the next slot.  In FP32 each u slot has a
// low part (set SET_UL) holding what the FP32 high part drops.
constexpr int NSLOT = 5;
enum { SET_UH = 0, SET_D = 5, SET_WORK = 10, SET_BH = 11, SET_UL = 12, SET_BL = 17 };
inline int nsets(bool lo) { return lo ? 18 : 12; }

template <typename T>
T* field_ptr(fftm_problem* p, int set, int q) {
  return reinterpret_cast<T*>(p->fields) + ((long long)set * 3 + q) * p->comp_stride;
}
template <typename T>
void set_ptrs(fftm_problem* p, int set, T* out[3]) {
  for (int q = 0; q < 3; ++q) out[q] = field_ptr<T>(p, set, q);
}

int ev_get(fftm_problem* p) {
  if (p->ev_free.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    p->ev.push_back(e);
    return (int)p->ev.size() - 1;
  }
  const int i = p->ev_free.back();
  p->ev_free.pop_back();
  return i;
}

// Brackets the launches of one category with two events when profiling is on.
// Device allocations of a problem: from the caller's workspace when it gave one (a bump
// allocator, 256-byte aligned; FFTM_E_NOMEM when it is exhausted), else cudaMalloc.  Memory of
// the workspace is released with the problem, never piecewise.
static cudaError_t dev_alloc(fftm_problem* p, void** ptr, size_t bytes) {
  if (!p->arena) return cudaMalloc(ptr, bytes);
  const size_t at = (p->arena_used + 255) & ~(size_t)255;
  if (at > p->arena_size || bytes > p->arena_size - at) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  *ptr = p->arena + at;
  p->arena_used = at + bytes;
  return cudaSuccess;
}

static void dev_free(fftm_problem* p, void* ptr) {
  if (!ptr) return;
  if (p->arena && static_cast<char*>(ptr) >= p->arena && static_cast<char*>(ptr) < p->arena + p->arena_size) return;
  cudaFree(ptr);
}

struct ProfScope {
  fftm_problem* p;
  int cat, a = -1;
  ProfScope(fftm_problem* p_, int c) : p(p_), cat(c) {
    if (p->prof && (a = ev_get(p)) >= 0) cudaEventRecord(p->ev[a], p->ctx->stream);
  }
  ~ProfScope() {
    if (a < 0) return;
    const int b = ev_get(p);
    if (b < 0) return;
    cudaEventRecord(p->ev[b], p->ctx->stream);
    p->pending.push_back({cat, a, b, p->prof_m, p->prof_post});
  }
};

// Accumulate the elapsed times of completed event pairs (call after a stream sync).  In a
// device-decided step, launches enqueued past the iteration the step stopped at did no work:
// with m_last >= 0 only the pairs of iterations up to it count (for the last iteration, only
// its residual and check).
void prof_flush(fftm_problem* p, int m_last = -1) {
  for (const auto& e : p->pending) {
    float ms = 0.f;
    const bool count = m_last < 0 || e.m < 0 || e.m < m_last || (e.m == m_last && !e.post);
    if (count && cudaEventElapsedTime(&ms, p->ev[e.a], p->ev[e.b]) == cudaSuccess) {
      p->prof_ms[e.cat] += ms;
      p->prof_cnt[e.cat] += 1;
    }
    p->ev_free.push_back(e.a);
    p->ev_free.push_back(e.b);
  }
  p->pending.clear();
}

template <typename T>
const typename V2<T>::t* tptr_v2(fftm_problem* p, size_t off) {
  return reinterpret_cast<const typename V2<T>::t*>(reinterpret_cast<char*>(p->tables) + off);
}
template <typename T>
const T* tptr(fftm_problem* p, size_t off) {
  return reinterpret_cast<const T*>(reinterpret_cast<char*>(p->tables) + off);
}

template <typename T>
AxisPlan<T> dev_plan(fftm_problem* p, int q, int a) {
  const HostPlan& h = p->plans[q][a];
  AxisPlan<T> d;
  d.kind = h.kind;
  d.n = h.n;
  d.lo = h.lo;
  d.L = h.L;
  d.M = h.M;
  d.nst = (int)h.radix.size();
  for (int s = 0; s < MAX_STAGES; ++s) d.radix[s] = s < d.nst ? h.radix[s] : 1;
  d.perm = reinterpret_cast<const int16_t*>(reinterpret_cast<char*>(p->tables) + p->off_perm[q][a]);
  d.tw = tptr_v2<T>(p, p->off_tw[q][a]);
  d.qw = tptr_v2<T>(p, p->off_qw[q][a]);
  return d;
}

double axis_norm(fftm_problem* p, int q, int a) {
  const int k = p->kind[q][a];
  return (k == K_DFT ? 1.0 : 2.0) * p->n[a];
}

template <typename T>
PassParams<T> pass_params(fftm_problem* p, int axis, int inverse, int fused, int in_set, int out_set) {
  PassParams<T> P;
  std::memset(&P, 0, sizeof(P));
  for (int q = 0; q < 3; ++q) {
    P.in[q] = field_ptr<T>(p, in_set, q);
    P.out[q] = field_ptr<T>(p, out_set, q);
    P.plan[q] = dev_plan<T>(p, q, axis);
    P.scale[q] = T(1);
  }
  P.axis = axis;
  for (int a = 0; a < 3; ++a) P.N[a] = p->N[a];
  P.stride[0] = 1;
  P.stride[1] = p->sy;
  P.stride[2] = p->sz;
  P.inverse = inverse;
  P.fused = fused;
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) {
      P.S2[q][a] = tptr<T>(p, p->off_S2[q][a]);
      P.C2[q][a] = tptr<T>(p, p->off_C2[q][a]);
      P.flo[q][a] = p->plans[q][a].lo;
      P.fL[q][a] = p->plans[q][a].L;
    }
  for (int a = 0; a < 3; ++a) P.hf[a] = T(4.0 / (p->h[a] * p->h[a]));
  const double lam0 = p->desc.green == FFTM_GREEN_MU0 ? 0.0 : p->desc.lambda0;
  P.two_mu0 = T(2.0 * p->desc.mu0);
  P.lam0 = T(lam0);
  P.tetra = p->tetra;
  for (int q = 0; q < 3; ++q) P.gscale[q] = T(1.0 / (axis_norm(p, q, 0) * axis_norm(p, q, 1) * axis_norm(p, q, 2)));
  P.stop = p->stop;
  return P;
}

template <typename T>
int launch_pp(fftm_problem* p, const PassParams<T>& P, int axis) {
  ProfScope ps(p, axis == 0 ? FFTM_KCAT_PASS_X : (axis == 1 ? FFTM_KCAT_PASS_Y : FFTM_KCAT_PASS_Z));
  CU(launch_pass<T>(P, p->maxM[axis], p->maxL[axis], p->n[axis], p->ctx->stream));
  p->launches++;
  return FFTM_OK;
}

template <typename T>
int run_pass(fftm_problem* p, int axis, int inverse, int fused, int in_set, int out_set, bool normalise) {
  PassParams<T> P = pass_params<T>(p, axis, inverse, fused, in_set, out_set);
  if (normalise)
    for (int q = 0; q < 3; ++q) P.scale[q] = T(1.0 / axis_norm(p, q, axis));
  return launch_pp<T>(p, P, axis);
}

TcPassParams tc_params(fftm_problem* p, int axis, int inverse, int fused, int in_set, int out_set) {
  TcPassParams P;
  std::memset(&P, 0, sizeof(P));
  const char* base = reinterpret_cast<const char*>(p->tcmat);
  for (int q = 0; q < 3; ++q) {
    P.in[q] = field_ptr<float>(p, in_set, q);
    P.out[q] = field_ptr<float>(p, out_set, q);
    P.lo[q] = p->plans[q][axis].lo;
    P.L[q] = p->plans[q][axis].L;
    P.Kp[q] = p->tcKp[q][axis];
    P.A[q] = reinterpret_cast<const uint16_t*>(base + (inverse ? p->off_tci[q][axis] : p->off_tcf[q][axis]));
    P.A2[q] = reinterpret_cast<const uint16_t*>(base + p->off_tci[q][axis]);
    P.scale[q] = 1.f;
    for (int a = 0; a < 3; ++a) {
      P.S2[q][a] = tptr<float>(p, p->off_S2[q][a]);
      P.C2[q][a] = tptr<float>(p, p->off_C2[q][a]);
      P.flo[q][a] = p->plans[q][a].lo;
      P.fL[q][a] = p->plans[q][a].L;
    }
    P.gscale[q] = 1.f;  // the inverse matrices carry the normalisation
  }
  P.axis = axis;
  for (int a = 0; a < 3; ++a) {
    P.N[a] = p->N[a];
    P.hf[a] = (float)(4.0 / (p->h[a] * p->h[a]));
  }
  P.stride[0] = 1;
  P.stride[1] = p->sy;
  P.stride[2] = p->sz;
  P.fused = fused;
  const double lam0 = p->desc.green == FFTM_GREEN_MU0 ? 0.0 : p->desc.lambda0;
  P.two_mu0 = (float)(2.0 * p->desc.mu0);
  P.lam0 = (float)lam0;
  P.tetra = p->tetra;
  P.err = p->tc_err;
  P.stop = p->stop;
  return P;
}

int launch_tc(fftm_problem* p, const TcPassParams& P) {
  ProfScope ps(p, P.axis == 0 ? FFTM_KCAT_PASS_X : (P.axis == 1 ? FFTM_KCAT_PASS_Y : FFTM_KCAT_PASS_Z));
  CU(launch_pass_tc(P, p->ctx->stream));
  p->launches++;
  return FFTM_OK;
}

// One TF32 tensor-core pass along `axis`: mode 0 plain (scale 1; the inverse matrices carry
// the normalisation), 1 x inverse accumulated onto a base field, 2 z forward times the Green
// factor.
TfPassParams tf_params(fftm_problem* p, int axis, int inverse, int mode, int in_set, int out_set) {
  TfPassParams P;
  std::memset(&P, 0, sizeof(P));
  const char* base = reinterpret_cast<const char*>(p->tcmat);
  for (int q = 0; q < 3; ++q) {
    P.in[q] = field_ptr<float>(p, in_set, q);
    P.out[q] = field_ptr<float>(p, out_set, q);
    P.lo[q] = p->plans[q][axis].lo;
    P.L[q] = p->plans[q][axis].L;
    P.Kp[q] = p->tcKp[q][axis];
    P.Kn[q] = p->tcKn[q][axis];
    P.xrow[q] = p->tcx[q][axis]
                    ? reinterpret_cast<const float*>(base + (inverse ? p->off_tcxi[q][axis] : p->off_tcxf[q][axis]))
                    : nullptr;
    P.A[q] = reinterpret_cast<const float*>(base + (inverse ? p->off_tci[q][axis] : p->off_tcf[q][axis]));
    P.scale[q] = 1.f;
    for (int a = 0; a < 3; ++a) {
      P.S2[q][a] = tptr<float>(p, p->off_S2[q][a]);
      P.C2[q][a] = tptr<float>(p, p->off_C2[q][a]);
      P.flo[q][a] = p->plans[q][a].lo;
      P.fL[q][a] = p->plans[q][a].L;
    }
    P.gscale[q] = 1.f;
  }
  P.axis = axis;
  P.mode = mode;
  for (int a = 0; a < 3; ++a) {
    P.N[a] = p->N[a];
    P.hf[a] = (float)(4.0 / (p->h[a] * p->h[a]));
  }
  P.stride[0] = 1;
  P.stride[1] = p->sy;
  P.stride[2] = p->sz;
  const double lam0 = p->desc.green == FFTM_GREEN_MU0 ? 0.0 : p->desc.lambda0;
  P.two_mu0 = (float)(2.0 * p->desc.mu0);
  P.lam0 = (float)lam0;
  P.tetra = p->tetra;
  P.err = p->tc_err;
  P.stop = p->stop;
  return P;
}

int launch_tf(fftm_problem* p, const TfPassParams& P) {
  ProfScope ps(p, P.axis == 0 ? FFTM_KCAT_PASS_X : (P.axis == 1 ? FFTM_KCAT_PASS_Y : FFTM_KCAT_PASS_Z));
  CU(launch_pass_tf32(P, p->ctx->stream));
  p->launches++;
  return FFTM_OK;
}

template <typename T>
ResParams<T> res_params(fftm_problem* p, int slot, T* D_base, T* p_base) {
  ResParams<T> R;
  std::memset(&R, 0, sizeof(R));
  const bool lo = p->esz == 4;
  for (int q = 0; q < 3; ++q) {
    R.u[q] = field_ptr<T>(p, SET_UH + slot, q);
    R.ulo[q] = lo ? field_ptr<T>(p, SET_UL + slot, q) : nullptr;
    R.D[q] = D_base ? D_base + q * p->comp_stride : field_ptr<T>(p, SET_D + slot, q);
    R.p[q] = p_base ? p_base + q * p->comp_stride : nullptr;
  }
  R.phase = p->phase;
  R.law_id = p->law_id;
  R.law_c = reinterpret_cast<const T*>(p->law_c);
  R.law_m = reinterpret_cast<const T*>(p->law_m);
  for (int a = 0; a < 3; ++a) {
    R.n[a] = p->n[a];
    R.N[a] = p->N[a];
    R.periodic[a] = p->periodic[a];
    R.wdiv[a] = T(0.25 / p->h[a]);
    R.wgrad[a] = T((p->tetra ? 0.5 : 0.25) / p->h[a]);
  }
  R.sy = p->sy;
  R.sz = p->sz;
  R.nsy = p->sy;
  R.nsz = p->sz;
  R.vy = p->n[0];
  R.vz = (long long)p->n[0] * p->n[1];
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < 3; ++q) R.Gs[i * 3 + q] = T(p->load.A[q][i]);  // G*_iq = d u*_q / d x_i
  const double lam0 = p->desc.green == FFTM_GREEN_MU0 ? 0.0 : p->desc.lambda0;
  R.lam0 = T(lam0);
  R.two_mu0 = T(2.0 * p->desc.mu0);
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) {
      R.sgn[q][a][0] = p->sgn[q][a][0];
      R.sgn[q][a][1] = p->sgn[q][a][1];
      R.lo[q][a] = p->lo[q][a];
      R.hi[q][a] = p->hi[q][a];
    }
  R.partial = p->partial;
  R.stop = p->stop;
  R.two_pass = p->res_two_pass > 0 ? 1 : 0;
  R.fused_fy = p->res_fy;
  R.vs = reinterpret_cast<T*>(p->vs);
  R.sym = p->sym;
  R.state = reinterpret_cast<T*>(p->state);
  R.nst = p->nst;
  R.slaw = p->slaw;
  R.c0 = p->c0;
  R.quad = 0;
  R.dquad = 0;
  for (int q = 0; q < 3; ++q) {
    for (int k = 0; k < 6; ++k) {
      R.Qc[q][k] = T(p->load.Q[q][k]);
      R.quad |= p->load.Q[q][k] != 0.0;
      const double dq = p->load.Q[q][k] - p->load_n.Q[q][k];
      R.dQ[q][k] = T(dq);
      R.dquad |= dq != 0.0;
    }
    R.un[q] = p->un ? reinterpret_cast<const T*>(p->un) + q * p->comp_stride : nullptr;
    R.unlo[q] = (p->un && lo) ? reinterpret_cast<const T*>(p->un) + (3 + q) * p->comp_stride : nullptr;
  }
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < 3; ++q) R.dGs[i * 3 + q] = T(p->load.A[q][i] - p->load_n.A[q][i]);
  for (int a = 0; a < 3; ++a) R.hh[a] = T(p->h[a]);
  R.traction = 0;
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < 2; ++f)
      for (int q = 0; q < 3; ++q) {
        R.tr[a][f][q] = T(p->load.T[a][f][q]);
        R.traction |= p->load.T[a][f][q] != 0.0;
      }
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < 2; ++f) {
      R.tface[a][f] = reinterpret_cast<const T*>(p->tface[a][f]);
      R.tface_n[a][f] = nullptr;
      R.traction |= p->tface[a][f] != nullptr;
    }
  for (int q = 0; q < 3; ++q) {
    R.us[q] = p->ustar ? reinterpret_cast<const T*>(p->ustar) + q * p->comp_stride : nullptr;
    R.us_n[q] = p->ustar_n ? reinterpret_cast<const T*>(p->ustar_n) + q * p->comp_stride : nullptr;
  }
  return R;
}

// Parameters whose u^f and u* are those of the last commit (state conversion).
template <typename T>
ResParams<T> commit_params(fftm_problem* p) {
  ResParams<T> R = res_params<T>(p, p->cur, nullptr, nullptr);
  if (p->commit_pending) R.state = reinterpret_cast<T*>(p->state_next);
  for (int q = 0; q < 3; ++q) {
    R.u[q] = R.un[q];
    R.ulo[q] = R.unlo[q];
  }
  R.quad = 0;
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < 6; ++k) {
      R.Qc[q][k] = T(p->load_n.Q[q][k]);
      R.quad |= p->load_n.Q[q][k] != 0.0;
    }
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < 3; ++q) R.Gs[i * 3 + q] = T(p->load_n.A[q][i]);
  return R;
}

// ---- launch-shape tuning ----------------------------------------------------------------
// Where a row of the path has several implementations with the same per-element arithmetic,
// the library times them on the problem's own data the first time a problem of that shape
// runs, keeps the fastest, and records the choice in a process-wide table keyed by the shape
// (fftm_tuning_table prints it).
std::mutex g_tune_mu;
std::map<std::string, std::string> g_tune_table;  // key -> "choice (times)"
std::map<std::string, int> g_tune_choice;

std::string residual_key(const fftm_problem* p) {
  char b[160];
  std::snprintf(b, sizeof(b), "residual %s %s %dx%dx%d %c%c%c", p->esz == 8 ? "fp64" : "fp32",
                p->tetra ? "TETRA2" : "HEX1", p->n[0], p->n[1], p->n[2], p->periodic[0] ? 'P' : 'B',
                p->periodic[1] ? 'P' : 'B', p->periodic[2] ? 'P' : 'B');
  return b;
}

// Milliseconds per launch of the residual in the given form (3 launches after one warm-up).
template <typename T>
double time_residual(fftm_problem* p, int slot, int two_pass, int fy) {
  ResParams<T> R = res_params<T>(p, slot, nullptr, nullptr);
  R.two_pass = two_pass;
  R.fused_fy = fy;
  cudaStream_t s = p->ctx->stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.0;
  }
  double ms = -1.0;
  if (launch_residual<T>(R, p->tetra, false, s, nullptr) == cudaSuccess) {
    cudaEventRecord(e0, s);
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i) ok = launch_residual<T>(R, p->tetra, false, s, nullptr) == cudaSuccess;
    cudaEventRecord(e1, s);
    float t = 0.f;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
      ms = t / 3.0;
  }
  p->launches += 8;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

// The residual's form: one pass with a tile of 8 or 16 voxel rows, or two passes; as
// requested, else the fastest measured for the problem's grid shape (once per process).
template <typename T>
int resolve_residual_form(fftm_problem* p, int slot) {
  ResParams<T> R = res_params<T>(p, slot, nullptr, nullptr);
  const bool one_ok = residual_one_pass<T>(R);
  if (!one_ok || p->res_passes == 2) {
    p->res_two_pass = 1;
    return FFTM_OK;
  }
  if (p->res_passes == 1 && p->res_tile != 0) {
    p->res_two_pass = 0;
    p->res_fy = p->res_tile;
    return FFTM_OK;
  }
  const std::string key = residual_key(p);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_choice.find(key);
    if (it != g_tune_choice.end()) {
      const int c = it->second;  // 0: one pass, fy 8; 1: one pass, fy 16; 2: two passes
      p->res_two_pass = (p->res_passes == 1) ? 0 : (c == 2 ? 1 : 0);
      p->res_fy = c == 1 ? 16 : 8;
      return FFTM_OK;
    }
  }
  const double t8 = time_residual<T>(p, slot, 0, 8), t16 = time_residual<T>(p, slot, 0, 16);
  const double t2 = p->res_passes == 1 ? -1.0 : time_residual<T>(p, slot, 1, 8);
  CU(cudaGetLastError());
  int c = 0;
  double best = t8;
  if (t16 >= 0.0 && (best < 0.0 || t16 < best)) c = 1, best = t16;
  if (t2 >= 0.0 && (best < 0.0 || t2 < best)) c = 2, best = t2;
  static const char* names[3] = {"one pass, 8-row tiles", "one pass, 16-row tiles", "two passes"};
  char b[200];
  std::snprintf(b, sizeof(b), "%s (one pass 8 rows %.4f ms, 16 rows %.4f ms; two passes %.4f ms)", names[c], t8, t16,
                t2);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_choice[key] = c;
    g_tune_table[key] = b;
  }
  p->res_two_pass = c == 2 ? 1 : 0;
  p->res_fy = c == 1 ? 16 : 8;
  return FFTM_OK;
}

// a1-a4: D (into the D slot of `slot`, or the test buffers) and the two norms.  solver_form:
// the solver's residual kernels (one pass where the form allows it, no p), D into the test
// buffer, no convergence test (FFTM_OP_RESIDUAL with the one-pass form forced).
template <typename T>
int run_residual(fftm_problem* p, int slot, bool test_outputs, bool solver_form = false) {
  if (!test_outputs && p->res_two_pass < 0) {
    int rc = resolve_residual_form<T>(p, slot);
    if (rc) return rc;
  }
  T* D = nullptr;
  T* pp = nullptr;
  if (test_outputs || solver_form) {
    if (!p->Dbuf) {
      DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->Dbuf), 3 * p->comp_stride * sizeof(T)));
      CU(cudaMemsetAsync(p->Dbuf, 0, 3 * p->comp_stride * sizeof(T), p->ctx->stream));
    }
    D = reinterpret_cast<T*>(p->Dbuf);
  }
  if (test_outputs) {
    pp = field_ptr<T>(p, SET_WORK, 0);
    if (!p->vs_test) {
      const size_t b = (size_t)(p->tetra ? 2 : 1) * ((p->sym ? 6 : 9) + 9) * p->nvox * sizeof(T);
      DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->vs_test), b));
    }
  }
  ResParams<T> R = res_params<T>(p, slot, D, pp);
  if (test_outputs) R.vs = reinterpret_cast<T*>(p->vs_test);
  if (!test_outputs && p->committed) {  // incremental form from the last commit
    R.inc = 1;
    for (int q = 0; q < 3; ++q) R.Dn[q] = reinterpret_cast<const T*>(p->Dn) + q * p->comp_stride;
    R.traction = 0;  // D_n holds the committed tractions' share: only their change enters
    for (int a = 0; a < 3; ++a)
      for (int f = 0; f < 2; ++f)
        for (int q = 0; q < 3; ++q) {
          const double dt = p->load.T[a][f][q] - p->load_n.T[a][f][q];
          R.tr[a][f][q] = T(dt);
          R.traction |= dt != 0.0;
        }
    for (int a = 0; a < 3; ++a)
      for (int f = 0; f < 2; ++f) {
        R.tface_n[a][f] = reinterpret_cast<const T*>(p->tface_n[a][f]);
        R.traction |= p->tface[a][f] != nullptr || p->tface_n[a][f] != nullptr;
      }
  }
  int blocks = 0;
  ProfScope ps(p, test_outputs ? FFTM_KCAT_OTHER : FFTM_KCAT_RESIDUAL);
  CU(launch_residual<T>(R, p->tetra, test_outputs, p->ctx->stream, &blocks));
  CU(launch_reduce_norms(p->partial, blocks, 2, p->dscal, p->ctx->stream, p->stop));
  p->launches += 2;
  if (p->stop && !test_outputs && !solver_form) {  // the convergence test on the device
    CU(launch_check(p->dscal, p->dctl, p->derr, p->desc.tol, p->desc.max_iter, p->h[0], p->ctx->stream));
    p->launches += 1;
  }
  return FFTM_OK;
}

// a6-a8: out = base - Gamma(in) (base may be absent: out = Gamma(in)).  The
// first pass reads `in_set`, the rest work in place on WORK; the z pass runs
// forward z, the Green factor and inverse z in one kernel.
template <typename T>
C0Params<T> c0_params(fftm_problem* p, bool normalised_inverse, bool negate) {
  C0Params<T> G;
  std::memset(&G, 0, sizeof(G));
  const T* tab = reinterpret_cast<const T*>(p->c0tab);
  size_t at = 0;
  for (int a = 0; a < 3; ++a) {
    G.N[a] = p->N[a];
    G.s[a] = tab + at;
    G.c[a] = tab + at + p->N[a];
    at += 2 * (size_t)p->N[a];
    G.hf[a] = T(2.0 / p->h[a]);
  }
  for (int q = 0; q < 3; ++q) {
    G.f[q] = field_ptr<T>(p, SET_WORK, q);
    for (int a = 0; a < 3; ++a) {
      G.lo[q][a] = p->plans[q][a].lo;
      G.hi[q][a] = p->plans[q][a].lo + p->plans[q][a].L;
    }
    G.tau[q] = p->kind[q][q] == K_DCT1 ? T(-1) : T(1);
    // the FFT inverse passes are unnormalised (the factor goes here); the tensor-core inverse
    // matrices carry it
    const double nrm = normalised_inverse ? 1.0 : axis_norm(p, q, 0) * axis_norm(p, q, 1) * axis_norm(p, q, 2);
    G.gscale[q] = T((negate ? -1.0 : 1.0) / nrm);
  }
  G.sy = p->sy;
  G.sz = p->sz;
  G.two_mu0 = T(2.0 * p->desc.mu0);
  G.beta = T(p->desc.lambda0 / (2.0 * p->desc.mu0 + p->desc.lambda0));
  G.lam0 = T(p->desc.lambda0);
  G.tetra = p->tetra;
  G.stop = p->stop;
  return G;
}

// a6-a8 with the C0 operator: the three forward passes, the coupled Green operator at every
// node position, the three inverse passes (the last one forms base - Gamma(in))
template <typename T>
int green_apply_c0(fftm_problem* p, int in_set, int base_set, int base_lo_set, int out_set, int out_lo_set,
                   bool negate) {
  int rc;
  const cudaStream_t s = p->ctx->stream;
  const bool tens = p->tf || p->tc;
  for (int a = 0; a < 3; ++a) {
    const int in = a == 0 ? in_set : SET_WORK;
    rc = p->tf ? launch_tf(p, tf_params(p, a, 0, 0, in, SET_WORK))
         : p->tc ? launch_tc(p, tc_params(p, a, 0, 0, in, SET_WORK))
                 : run_pass<T>(p, a, 0, 0, in, SET_WORK, false);
    if (rc) return rc;
  }
  {
    ProfScope ps(p, FFTM_KCAT_PASS_Z);
    CU(launch_green_c0<T>(c0_params<T>(p, tens, negate), s));
    p->launches++;
  }
  for (int a = 2; a >= 1; --a) {
    rc = p->tf ? launch_tf(p, tf_params(p, a, 1, 0, SET_WORK, SET_WORK))
         : p->tc ? launch_tc(p, tc_params(p, a, 1, 0, SET_WORK, SET_WORK))
                 : run_pass<T>(p, a, 1, 0, SET_WORK, SET_WORK, false);
    if (rc) return rc;
  }
  if (p->tf) {
    TfPassParams P = tf_params(p, 0, 1, base_set >= 0 ? 1 : 0, SET_WORK, out_set);
    if (base_set >= 0)
      for (int q = 0; q < 3; ++q) {
        P.base[q] = field_ptr<float>(p, base_set, q);
        P.base_lo[q] = base_lo_set >= 0 ? field_ptr<float>(p, base_lo_set, q) : nullptr;
        P.out_lo[q] = out_lo_set >= 0 ? field_ptr<float>(p, out_lo_set, q) : nullptr;
      }
    return launch_tf(p, P);
  }
  if (p->tc) {
    TcPassParams P = tc_params(p, 0, 1, 0, SET_WORK, out_set);
    if (base_set >= 0)
      for (int q = 0; q < 3; ++q) {
        P.base[q] = field_ptr<float>(p, base_set, q);
        P.base_lo[q] = base_lo_set >= 0 ? field_ptr<float>(p, base_lo_set, q) : nullptr;
        P.out_lo[q] = out_lo_set >= 0 ? field_ptr<float>(p, out_lo_set, q) : nullptr;
      }
    return launch_tc(p, P);
  }
  PassParams<T> P = pass_params<T>(p, 0, 1, 0, SET_WORK, out_set);
  if (base_set >= 0)
    for (int q = 0; q < 3; ++q) {
      P.base[q] = field_ptr<T>(p, base_set, q);
      P.base_lo[q] = base_lo_set >= 0 ? field_ptr<T>(p, base_lo_set, q) : nullptr;
      P.out_lo[q] = out_lo_set >= 0 ? field_ptr<T>(p, out_lo_set, q) : nullptr;
    }
  return launch_pp<T>(p, P, 0);
}

template <typename T>
int green_apply(fftm_problem* p, int in_set, int base_set, int base_lo_set, int out_set, int out_lo_set,
                bool negate) {
  int rc;
  if (p->c0) return green_apply_c0<T>(p, in_set, base_set, base_lo_set, out_set, out_lo_set, negate);
  if (p->tf) {
    if ((rc = launch_tf(p, tf_params(p, 0, 0, 0, in_set, SET_WORK)))) return rc;
    if ((rc = launch_tf(p, tf_params(p, 1, 0, 0, SET_WORK, SET_WORK)))) return rc;
    {
      TfPassParams P = tf_params(p, 2, 0, 2, SET_WORK, SET_WORK);
      if (negate)
        for (int q = 0; q < 3; ++q) P.gscale[q] = -1.f;
      if ((rc = launch_tf(p, P))) return rc;
    }
    if ((rc = launch_tf(p, tf_params(p, 2, 1, 0, SET_WORK, SET_WORK)))) return rc;
    if ((rc = launch_tf(p, tf_params(p, 1, 1, 0, SET_WORK, SET_WORK)))) return rc;
    TfPassParams P = tf_params(p, 0, 1, base_set >= 0 ? 1 : 0, SET_WORK, out_set);
    if (base_set >= 0)
      for (int q = 0; q < 3; ++q) {
        P.base[q] = field_ptr<float>(p, base_set, q);
        P.base_lo[q] = base_lo_set >= 0 ? field_ptr<float>(p, base_lo_set, q) : nullptr;
        P.out_lo[q] = out_lo_set >= 0 ? field_ptr<float>(p, out_lo_set, q) : nullptr;
      }
    return launch_tf(p, P);
  }
  if (p->tc) {
    if ((rc = launch_tc(p, tc_params(p, 0, 0, 0, in_set, SET_WORK)))) return rc;
    if ((rc = launch_tc(p, tc_params(p, 1, 0, 0, SET_WORK, SET_WORK)))) return rc;
    {
      TcPassParams P = tc_params(p, 2, 0, 1, SET_WORK, SET_WORK);
      if (negate)
        for (int q = 0; q < 3; ++q) P.gscale[q] = -1.f;
      if ((rc = launch_tc(p, P))) return rc;
    }
    if ((rc = launch_tc(p, tc_params(p, 1, 1, 0, SET_WORK, SET_WORK)))) return rc;
    TcPassParams P = tc_params(p, 0, 1, 0, SET_WORK, out_set);
    if (base_set >= 0)
      for (int q = 0; q < 3; ++q) {
        P.base[q] = field_ptr<float>(p, base_set, q);
        P.base_lo[q] = base_lo_set >= 0 ? field_ptr<float>(p, base_lo_set, q) : nullptr;
        P.out_lo[q] = out_lo_set >= 0 ? field_ptr<float>(p, out_lo_set, q) : nullptr;
      }
    return launch_tc(p, P);
  }
  if ((rc = run_pass<T>(p, 0, 0, 0, in_set, SET_WORK, false))) return rc;
  if ((rc = run_pass<T>(p, 1, 0, 0, SET_WORK, SET_WORK, false))) return rc;
  {
    PassParams<T> P = pass_params<T>(p, 2, 0, 1, SET_WORK, SET_WORK);
    if (negate)
      for (int q = 0; q < 3; ++q) P.gscale[q] = -P.gscale[q];
    if ((rc = launch_pp<T>(p, P, 2))) return rc;
  }
  if ((rc = run_pass<T>(p, 1, 1, 0, SET_WORK, SET_WORK, false))) return rc;
  PassParams<T> P = pass_params<T>(p, 0, 1, 0, SET_WORK, out_set);
  if (base_set >= 0)
    for (int q = 0; q < 3; ++q) {
      P.base[q] = field_ptr<T>(p, base_set, q);
      P.base_lo[q] = base_lo_set >= 0 ? field_ptr<T>(p, base_lo_set, q) : nullptr;
      P.out_lo[q] = out_lo_set >= 0 ? field_ptr<T>(p, out_lo_set, q) : nullptr;
    }
  return launch_pp<T>(p, P, 0);
}

double error_of(fftm_problem* p, double SD, double SP) {
  if (SP > 0.0) return p->h[0] * std::sqrt(SD / SP);
  return SD == 0.0 ? 0.0 : INFINITY;
}

// Normal-mixed loading (Sec. 3.2, Eq. NMBC1): strain components of u* (Voigt order 11,
// 22, 33, 23, 13, 12, bit k of the mask) adjusted after every residual so that the mean
// stress vanishes in them.  The paper gives no update rule; this one takes the
// increment -(C0_FF)^-1 <sigma>_F of the isotropic reference stiffness restricted to the
// free components (the normal ones couple through lambda0, the shear ones decouple).
constexpr int kVoigt[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
constexpr int kStatsBlocks = 152 * 2;  // blocks of the mean stress / strain reduction

void mixed_increment(const double sig[3][3], int mask, double lam0, double mu0, double d[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) d[i][j] = 0.0;
  int nn = 0, idx[3];
  double M[3][4];
  for (int k = 0; k < 3; ++k)
    if ((mask >> k) & 1) idx[nn++] = k;
  for (int r = 0; r < nn; ++r) {
    for (int c = 0; c < nn; ++c) M[r][c] = lam0 + (r == c ? 2.0 * mu0 : 0.0);
    M[r][nn] = -sig[idx[r]][idx[r]];
  }
  for (int c = 0; c < nn; ++c) {  // Gauss-Jordan; the matrix is symmetric positive definite
    for (int r = 0; r < nn; ++r) {
      if (r == c) continue;
      const double f = M[r][c] / M[c][c];
      for (int k = c; k <= nn; ++k) M[r][k] -= f * M[c][k];
    }
  }
  for (int r = 0; r < nn; ++r) d[idx[r]][idx[r]] = M[r][nn] / M[r][r];
  for (int k = 3; k < 6; ++k)
    if ((mask >> k) & 1) {
      const int i = kVoigt[k][0], j = kVoigt[k][1];
      d[i][j] = d[j][i] = -sig[i][j] / (2.0 * mu0);
    }
}

// ||<sigma>_F|| / ||<sigma>|| (tensor norms: both off-diagonal entries counted).
double mixed_error(const double sig[3][3], int mask) {
  double tot = 0.0, f = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) tot += sig[i][j] * sig[i][j];
  if (tot == 0.0) return 0.0;
  for (int k = 0; k < 6; ++k)
    if ((mask >> k) & 1) {
      const int i = kVoigt[k][0], j = kVoigt[k][1];
      f += sig[i][j] * sig[i][j] * (i == j ? 1.0 : 2.0);
    }
  return std::sqrt(f / tot);
}

// The update that follows the residual of iteration m (a5-a8): u^{m+1} into the next ring slot,
// either u^m - Gamma(D^m) or, on an Anderson iteration with a full history, the mix of the
// stored couples minus Gamma of the mixed residual.  In a device-decided step the launches
// carry the stop flag and the Anderson flag goes to the iteration the device checked last.
template <typename T>
int update_after(fftm_problem* p, int m, int cur0) {
  cudaStream_t s = p->ctx->stream;
  const bool lo = p->esz == 4;
  const int depth = p->desc.anderson_depth, period = p->desc.anderson_period;
  const long long cnt = p->comp_stride;
  const int sm = (cur0 + m) % NSLOT, sn = (cur0 + m + 1) % NSLOT;
  // couples k = m - depth + 1 .. m (k >= 1) are in slots (cur0 + k) % NSLOT
  const int have = std::min(m, depth);
  const bool accel = depth > 0 && (m % period == period - 1) && have == depth;
  if (accel) {
    const T* Ds[4][3];
    const T* uh[4][3];
    const T* ul[4][3];
    for (int j = 0; j < 4; ++j) {
      const int k = m - depth + 1 + std::min(j, depth - 1);
      const int sk = (cur0 + k) % NSLOT;
      for (int q = 0; q < 3; ++q) {
        Ds[j][q] = field_ptr<T>(p, SET_D + sk, q);
        uh[j][q] = field_ptr<T>(p, SET_UH + sk, q);
        ul[j][q] = lo ? field_ptr<T>(p, SET_UL + sk, q) : nullptr;
      }
    }
    {
      const int gb = gram_blocks(cnt);
      ProfScope ps(p, FFTM_KCAT_ANDERSON);
      CU(launch_gram<T>(Ds, depth, cnt, p->partial, gb, s, p->stop));
      if (p->stop)
        CU(launch_anderson_solve(p->partial, gb, depth, 1e-8, p->dscal + 2, p->dint, s, p->dctl));
      else
        CU(launch_anderson_solve(p->partial, gb, depth, 1e-8, p->dscal + 2, p->dint + m, s));
      T* work[3];
      T* bh[3];
      T* bl[3];
      set_ptrs<T>(p, SET_WORK, work);
      set_ptrs<T>(p, SET_BH, bh);
      if (lo) set_ptrs<T>(p, SET_BL, bl);
      CU(launch_combine<T>(work, bh, lo ? bl : nullptr, Ds, uh, ul, depth, p->dscal + 2, cnt, s, p->stop));
      p->launches += 3;
    }
    return green_apply<T>(p, SET_WORK, SET_BH, lo ? SET_BL : -1, SET_UH + sn, lo ? SET_UL + sn : -1, true);
  }
  return green_apply<T>(p, SET_D + sm, SET_UH + sm, lo ? SET_UL + sm : -1, SET_UH + sn, lo ? SET_UL + sn : -1,
                        true);
}

// A load step whose convergence test runs on the device (every load without a normal-mixed
// part): the host enqueues iterations in chunks (residual, reduction, k_check, update), every
// launch after the test stops the step does nothing, and the host waits once per chunk.
// Returns the last checked iteration in *m_out and the stop code in *stop_out.
constexpr int kDevChunk = 4;

// Device-decided steps replayed from CUDA graphs.  The launches of iteration m depend on m only
// through the slot ring (m mod NSLOT) and the Anderson gate (m mod period, and whether `depth`
// couples exist yet), so iterations [G, 2G) with G = lcm(NSLOT, period) repeat for every later
// block of G.  Two graphs are captured per load step (their kernel arguments hold the load):
// iterations [0, G) and [G, 2G); the second is replayed until the stop flag is set.  Kernels
// replayed past the stop return at once.  FFTM_E_UNSUPPORTED: the capture failed (the caller
// falls back to enqueueing the iterations one by one).
template <typename T>
int graph_loop(fftm_problem* p, int cur0, int* stop_out, int* mlast_out) {
  cudaStream_t s = p->ctx->stream;
  const int max_iter = p->desc.max_iter;
  const int depth = p->desc.anderson_depth, period = std::max(1, p->desc.anderson_period);
  int G = NSLOT;
  if (depth > 0) {
    int a = NSLOT, b = period;
    while (b) { const int t = a % b; a = b; b = t; }
    G = NSLOT / a * period;
    while (G < depth) G += NSLOT / a * period;
  }
  cudaGraphExec_t ex[2] = {nullptr, nullptr};
  long long ncap[2] = {0, 0};
  int rc = FFTM_OK;
  for (int k = 0; k < 2 && !rc; ++k) {
    const long long before = p->launches;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      rc = FFTM_E_UNSUPPORTED;
      break;
    }
    int irc = FFTM_OK;
    for (int m = k * G; m < (k + 1) * G && !irc; ++m) {
      irc = run_residual<T>(p, (cur0 + m) % NSLOT, false);
      if (!irc) irc = update_after<T>(p, m, cur0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    ncap[k] = p->launches - before;
    p->launches = before;
    if (irc || e != cudaSuccess || !g || cudaGraphInstantiate(&ex[k], g, 0) != cudaSuccess) rc = FFTM_E_UNSUPPORTED;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
  }
  int stop = 0, mlast = 0;
  int* hctl = reinterpret_cast<int*>(p->hpin + 40);
  for (int m0 = 0; !rc && m0 <= max_iter; m0 += G) {
    const int k = m0 == 0 ? 0 : 1;
    if (cudaGraphLaunch(ex[k], s) != cudaSuccess ||
        cudaMemcpyAsync(hctl, p->dctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = set_err(FFTM_E_CUDA, std::string("graph replay: ") + cudaGetErrorString(cudaGetLastError()));
      break;
    }
    p->launches += ncap[k];
    stop = hctl[0];
    mlast = hctl[2];
    if (stop) break;
  }
  for (int k = 0; k < 2; ++k)
    if (ex[k]) cudaGraphExecDestroy(ex[k]);
  *stop_out = stop;
  *mlast_out = mlast;
  return rc;
}

template <typename T>
int device_loop(fftm_problem* p, int cur0, int* m_out, int* stop_out) {
  cudaStream_t s = p->ctx->stream;
  const int max_iter = p->desc.max_iter;
  if (p->derr_len < max_iter + 1) {
    if (p->derr) dev_free(p, p->derr);
    p->derr = nullptr;
    DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->derr), (max_iter + 1) * sizeof(double)));
    p->derr_len = max_iter + 1;
  }
  if (!p->dctl) DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->dctl), 4 * sizeof(int)));
  CU(cudaMemsetAsync(p->dctl, 0, 4 * sizeof(int), s));
  if (p->res_two_pass < 0) {  // the residual's form is measured before anything is enqueued
    int rc = resolve_residual_form<T>(p, cur0 % NSLOT);
    if (rc) return rc;
  }
  int* hctl = reinterpret_cast<int*>(p->hpin + 40);
  int stop = 0, mlast = 0;
  p->stop = p->dctl;
  int rc = FFTM_OK;
  if (p->graph && !p->prof) {
    const int grc = graph_loop<T>(p, cur0, &stop, &mlast);
    if (grc != FFTM_E_UNSUPPORTED) {  // else: the stream could not be captured, enqueue as usual
      p->stop = nullptr;
      if (grc) return grc;
      p->last_iters = mlast;
      *m_out = mlast;
      *stop_out = stop;
      return FFTM_OK;
    }
    CU(cudaMemsetAsync(p->dctl, 0, 4 * sizeof(int), s));
  }
  // chunks of kDevChunk iterations; near the iteration count of the previous step (a repeated or
  // similar load) the chunks shrink to one, so a step that stops there enqueues no idle work
  for (int m0 = 0, K = kDevChunk; m0 <= max_iter && !rc; m0 += K) {
    K = kDevChunk;
    if (p->last_iters >= 0 && m0 <= p->last_iters + 1) K = std::max(1, std::min(kDevChunk, p->last_iters - m0));
    for (int m = m0; m < m0 + K && m <= max_iter && !rc; ++m) {
      p->prof_m = m;
      p->prof_post = 0;
      rc = run_residual<T>(p, (cur0 + m) % NSLOT, false);
      if (rc || m >= max_iter) break;
      p->prof_post = 1;
      rc = update_after<T>(p, m, cur0);
    }
    if (rc) break;
    if (cudaMemcpyAsync(hctl, p->dctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = set_err(FFTM_E_CUDA, std::string("device-decided step: ") + cudaGetErrorString(cudaGetLastError()));
      break;
    }
    stop = hctl[0];
    mlast = hctl[2];
    prof_flush(p, stop ? mlast : -1);
    if (stop) break;
  }
  p->stop = nullptr;
  p->prof_m = -1;
  p->prof_post = 0;
  if (rc) return rc;
  p->last_iters = mlast;
  *m_out = mlast;
  *stop_out = stop;
  return FFTM_OK;
}

// Algorithm 1 for one load step.  The update of iteration m is
//   u^{m+1} = u^m - Gamma(D^m)                                 (plain step)
//   u^{m+1} = sum_k c_k u^k - Gamma(sum_k c_k D^k)             (Anderson step)
// which equals the paper's u^{m+1} = Gamma(p^m), p^m = div(R0 : grad u^m) - D^m,
// because Gamma inverts div(R0 : grad .) exactly on the transformed fields.
template <typename T>
int solve_step_t(fftm_problem* p, fftm_step_report* rep, double* err_hist, int* acc_hist, int hist_len) {
  cudaStream_t s = p->ctx->stream;
  const bool lo = p->esz == 4;
  const int depth = p->desc.anderson_depth, period = p->desc.anderson_period;
  const int max_iter = p->desc.max_iter;
  const long long cnt = p->comp_stride;
  if (p->dint_len < max_iter + 1) {
    if (p->dint) dev_free(p, p->dint);
    p->dint = nullptr;
    DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->dint), (max_iter + 1) * sizeof(int)));
    p->dint_len = max_iter + 1;
  }
  CU(cudaMemsetAsync(p->dint, 0, (max_iter + 1) * sizeof(int), s));
  if (p->commit_pending) {  // the previous step's commit becomes the state of this step
    std::swap(p->state, p->state_next);
    p->commit_pending = 0;
  }
  const int cur0 = p->cur;
  int m = 0, converged = 0;
  double err = 0.0;
  if (p->dev_loop && !p->load.mixed) {
    int stop = 0;
    int rc = device_loop<T>(p, cur0, &m, &stop);
    if (rc) return rc;
    std::vector<double> eh(m + 1);
    CU(cudaMemcpy(eh.data(), p->derr, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    for (int i = 0; i <= m && err_hist && i < hist_len; ++i) err_hist[i] = eh[i];
    err = eh[m];
    p->cur = (cur0 + m) % NSLOT;
    if (stop == 2) return set_err(FFTM_E_DIVERGED, "non-finite equilibrium norm");
    converged = stop == 1;
  } else
  for (m = 0;; ++m) {
    const int sm = (cur0 + m) % NSLOT;
    int rc = run_residual<T>(p, sm, false);
    if (rc) return rc;
    const int mixed = p->load.mixed;
    if (mixed) {  // the mean stress of this iterate (voxel points)
      ResParams<T> R = res_params<T>(p, sm, nullptr, nullptr);
      ProfScope ps(p, FFTM_KCAT_OTHER);
      CU(launch_stats<T>(R, p->tetra, p->partial, kStatsBlocks, s));
      CU(launch_reduce_norms(p->partial, kStatsBlocks, 18, p->dscal + 16, s));
      p->launches += 2;
    }
    CU(cudaMemcpyAsync(p->hpin, p->dscal, (mixed ? 25 : 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    prof_flush(p);
    err = error_of(p, p->hpin[0], p->hpin[1]);
    if (err_hist && m < hist_len) err_hist[m] = err;
    p->cur = sm;
    // err is +inf while the stress is still zero under a non-zero residual (a load carried
    // only by tractions, first iteration): not converged; NaN or an infinite norm diverged
    if (std::isnan(err) || !std::isfinite(p->hpin[0]) || !std::isfinite(p->hpin[1]))
      return set_err(FFTM_E_DIVERGED, "non-finite equilibrium norm");
    double sig[3][3];
    double mix_err = 0.0;
    if (mixed) {
      const double npts = (double)p->nvox * (p->tetra ? 2 : 1);
      for (int i = 0; i < 3; ++i)
        for (int q = 0; q < 3; ++q)
          sig[i][q] = 0.5 * (p->hpin[16 + i * 3 + q] + p->hpin[16 + q * 3 + i]) / npts;
      mix_err = mixed_error(sig, mixed);
      if (!std::isfinite(mix_err)) return set_err(FFTM_E_DIVERGED, "non-finite mean stress");
    }
    if (err < p->desc.tol && mix_err < p->desc.tol) {
      converged = 1;
      break;
    }
    if (mixed && m < max_iter) {  // the free strain components of u* for the next residual
      double d[3][3];
      mixed_increment(sig, mixed, p->desc.lambda0, p->desc.mu0, d);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) p->load.A[i][j] += d[i][j];
    }
    if (m >= max_iter) break;
    rc = update_after<T>(p, m, cur0);
    if (rc) return rc;
  }
  // report
  std::vector<int> acc(m + 1, 0);
  CU(cudaMemcpyAsync(acc.data(), p->dint, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (p->load.mixed) {
    std::memcpy(p->mixed_A, p->load.A, sizeof(p->mixed_A));
    p->mixed_prev = p->load.mixed;
  }
  const int sb = kStatsBlocks;
  {
    ResParams<T> R = res_params<T>(p, p->cur, nullptr, nullptr);
    ProfScope ps(p, FFTM_KCAT_OTHER);
    CU(launch_stats<T>(R, p->tetra, p->partial, sb, s));
    CU(launch_reduce_norms(p->partial, sb, 18, p->dscal + 16, s));
    p->launches += 2;
  }
  CU(cudaMemcpyAsync(p->hpin + 16, p->dscal + 16, 18 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (converged && p->state) {  // a9: commit the internal variables of the converged step
    ResParams<T> R = res_params<T>(p, p->cur, nullptr, nullptr);
    ProfScope ps(p, FFTM_KCAT_OTHER);
    // J2 and logarithmic J2 are rate-independent: the return at the converged field from the committed state
    // gives back the converged stress, so it commits in place.  The rate-dependent crystal
    // plasticity law would slip further; its commit waits in state_next for the next step.
    if (p->slaw == 2) {
      CU(launch_commit<T>(R, p->tetra, reinterpret_cast<T*>(p->state_next), s));
      p->commit_pending = 1;
    } else {
      CU(launch_commit<T>(R, p->tetra, reinterpret_cast<T*>(p->state), s));
    }
    p->launches += 1;
  }
  if (converged && p->inc_ok) {
    for (int q = 0; q < 3; ++q) {
      T* un = reinterpret_cast<T*>(p->un);
      CU(cudaMemcpyAsync(un + q * cnt, field_ptr<T>(p, SET_UH + p->cur, q), cnt * sizeof(T),
                         cudaMemcpyDeviceToDevice, s));
      if (lo)
        CU(cudaMemcpyAsync(un + (3 + q) * cnt, field_ptr<T>(p, SET_UL + p->cur, q), cnt * sizeof(T),
                           cudaMemcpyDeviceToDevice, s));
    }
    p->load_n = p->load;
    if (p->ustar) {  // the u* field at the commit
      const size_t ub = 3 * (size_t)p->comp_stride * sizeof(T);
      if (!p->ustar_n) DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->ustar_n), ub));
      CU(cudaMemcpyAsync(p->ustar_n, p->ustar, ub, cudaMemcpyDeviceToDevice, s));
    } else if (p->ustar_n) {
      CU(cudaMemsetAsync(p->ustar_n, 0, 3 * (size_t)p->comp_stride * sizeof(T), s));
    }
    for (int a = 0; a < 3; ++a)  // the face traction fields at the commit
      for (int f = 0; f < 2; ++f) {
        if (!p->tface[a][f]) {
          dev_free(p, p->tface_n[a][f]);
          p->tface_n[a][f] = nullptr;
          continue;
        }
        const size_t nb = (size_t)3 * p->n[a == 0 ? 1 : 0] * p->n[a == 2 ? 1 : 2] * sizeof(T);
        if (!p->tface_n[a][f]) DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->tface_n[a][f]), nb));
        CU(cudaMemcpyAsync(p->tface_n[a][f], p->tface[a][f], nb, cudaMemcpyDeviceToDevice, s));
      }
    p->committed = 1;
    // D_n = div P_n evaluated afresh (plain form) so that rounding does not accumulate
    // from step to step through the incremental form
    ResParams<T> Rn = res_params<T>(p, p->cur, reinterpret_cast<T*>(p->Dn), nullptr);
    CU(launch_residual<T>(Rn, p->tetra, false, s, nullptr));
    p->launches += 2;
  }
  CU(cudaStreamSynchronize(s));
  prof_flush(p);
  std::memset(rep, 0, sizeof(*rep));
  rep->iterations = m;
  rep->converged = converged;
  rep->err = err;
  int nacc = 0;
  for (int i = 0; i <= m; ++i) {
    if (acc_hist && i < hist_len) acc_hist[i] = acc[i];
    nacc += acc[i];
  }
  rep->n_accelerated = nacc;
  if (p->tc || p->tf) {  // a tensor-core pass that gave up on a barrier leaves its result undefined
    int e = 0;
    CU(cudaMemcpy(&e, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      CU(cudaMemset(p->tc_err, 0, sizeof(int)));
      return set_err(FFTM_E_TIMEOUT, "a tensor-core transform pass timed out waiting for its MMAs");
    }
  }
  const double npts = (double)p->nvox * (p->tetra ? 2 : 1);
  static const int map6[6] = {0, 4, 8, 5, 2, 1};
  for (int c = 0; c < 6; ++c) rep->mean_P[c] = p->hpin[16 + map6[c]] / npts;
  for (int c = 0; c < 9; ++c) rep->mean_G[c] = p->hpin[16 + 9 + c] / npts;
  return converged ? FFTM_OK : FFTM_NOT_CONVERGED;
}

// The Lame pair a phase contributes to an automatic reference medium.
void phase_lame(const fftm_material& m, double* lam, double* mu) {
  const double* c = m.params;
  switch (m.law) {
    case FFTM_LAW_CUBIC_ELASTIC:
    case FFTM_LAW_SVK_CUBIC:
    case FFTM_LAW_CP_FCC:
      *lam = c[1];
      *mu = 0.5 * (c[2] + 0.5 * (c[0] - c[1]));
      return;
    case FFTM_LAW_NEO_HOOKE:
      *lam = c[1] - 2.0 * c[0] / 3.0;
      *mu = c[0];
      return;
    default:  // isotropic, J2, B0-linear, logarithmic J2: (lambda, mu) first
      *lam = c[0];
      *mu = c[1];
  }
}

// a copy of the descriptor with the reference medium resolved (FFTM_REF_AUTO)
int resolved_desc(const fftm_problem_desc* in, fftm_problem_desc* out) {
  if (!in) return set_err(FFTM_E_INVALID, "null descriptor");
  *out = *in;
  return fftm_host_reference_medium(in, &out->lambda0, &out->mu0);
}

int validate(const fftm_problem_desc* d) {
  if (!d) return set_err(FFTM_E_INVALID, "null descriptor");
  for (int a = 0; a < 3; ++a) {
    if (d->n[a] < 2 || d->n[a] > 8192) return set_err(FFTM_E_INVALID, "n must be in [2, 8192]");
    if (!(d->h[a] > 0.0)) return set_err(FFTM_E_INVALID, "h must be > 0");
  }
  if (!d->phase) return set_err(FFTM_E_INVALID, "phase map is null");
  if (d->n_phases < 1 || d->n_phases > 65535 || !d->materials)
    return set_err(FFTM_E_INVALID, "n_phases must be in [1, 65535] with a materials array");
  for (int i = 0; i < d->n_phases; ++i) {
    const int law = d->materials[i].law;
    if (law != FFTM_LAW_ISO_ELASTIC && law != FFTM_LAW_CUBIC_ELASTIC && law != FFTM_LAW_B0_LINEAR &&
        law != FFTM_LAW_J2_LINHARD && law != FFTM_LAW_SVK_CUBIC && law != FFTM_LAW_NEO_HOOKE &&
        law != FFTM_LAW_CP_FCC && law != FFTM_LAW_LOG_J2)
      return set_err(FFTM_E_INVALID, "unknown law");
    if (law == FFTM_LAW_LOG_J2) {
      const double* c = d->materials[i].params;
      if (!(c[1] > 0.0) || !(3.0 * c[0] + 2.0 * c[1] > 0.0) || !(c[2] > 0.0))
        return set_err(FFTM_E_INVALID, "logarithmic J2 needs mu > 0, 3 lambda + 2 mu > 0, sigma0 > 0");
    }
    if (law == FFTM_LAW_CP_FCC) {
      const double* c = d->materials[i].params;
      if (!(c[0] > 0 && c[1] > 0 && c[2] > 0 && c[3] > 0 && c[4] >= 1 && c[5] > 0 && c[6] >= c[5] && c[7] >= 0 &&
            c[8] > 0))
        return set_err(FFTM_E_INVALID,
                       "crystal plasticity needs C11, C12, C44, gdot0 > 0, n >= 1, tau0 > 0, tau_inf >= tau0, h0 >= 0, dt > 0");
    }
    if (law == FFTM_LAW_NEO_HOOKE && !(d->materials[i].params[0] > 0.0 && d->materials[i].params[1] > 0.0))
      return set_err(FFTM_E_INVALID, "Neo-Hookean needs mu > 0 and K > 0");
    if (law == FFTM_LAW_J2_LINHARD) {
      const double* c = d->materials[i].params;
      if (!(c[1] > 0.0) || !(3.0 * c[0] + 2.0 * c[1] > 0.0) || !(c[2] > 0.0) || !(c[3] >= 0.0))
        return set_err(FFTM_E_INVALID, "J2 needs mu > 0, 3 lambda + 2 mu > 0, sigma_y > 0, H >= 0");
    }
  }
  {
    bool j2 = false, cp = false, lj2 = false;
    for (int i = 0; i < d->n_phases; ++i) {
      j2 |= d->materials[i].law == FFTM_LAW_J2_LINHARD;
      cp |= d->materials[i].law == FFTM_LAW_CP_FCC;
      lj2 |= d->materials[i].law == FFTM_LAW_LOG_J2;
    }
    if ((int)j2 + (int)cp + (int)lj2 > 1)
      return set_err(FFTM_E_UNSUPPORTED, "phases of more than one law with internal variables (J2, crystal "
                                         "plasticity, logarithmic J2) in one problem");
  }
  for (int a = 0; a < 3; ++a) {
    int np = 0;
    for (int f = 0; f < 2; ++f)
      for (int q = 0; q < 3; ++q) {
        const int b = d->bc[a][f][q];
        if (b != FFTM_BC_PERIODIC && b != FFTM_BC_DIRICHLET && b != FFTM_BC_NEUMANN)
          return set_err(FFTM_E_INVALID, "bad bc value");
        np += (b == FFTM_BC_PERIODIC);
      }
    if (np != 0 && np != 6)
      return set_err(FFTM_E_INVALID, "a periodic axis must be periodic on both faces for every component");
  }
  if (d->scheme != FFTM_HEX1 && d->scheme != FFTM_TETRA2) return set_err(FFTM_E_INVALID, "bad scheme");
  if (d->green != FFTM_GREEN_B0 && d->green != FFTM_GREEN_MU0 && d->green != FFTM_GREEN_C0)
    return set_err(FFTM_E_INVALID, "bad green");
  if (d->green == FFTM_GREEN_C0) {  // Sec. 2.6.1: normal-mixed BCs (Eq. SGO_BCs), as built here
    for (int a = 0; a < 3; ++a)
      for (int q = 0; q < 3; ++q) {
        const int b0 = d->bc[a][0][q], b1 = d->bc[a][1][q];
        if (b0 == FFTM_BC_PERIODIC || b0 != b1)
          return set_err(FFTM_E_UNSUPPORTED, "the C0 Green operator needs non-periodic axes with the same "
                                             "condition on both faces");
        if (q != a && b0 == d->bc[a][0][a])
          return set_err(FFTM_E_UNSUPPORTED, "the C0 Green operator needs normal-mixed conditions: on each axis "
                                             "the normal component Dirichlet and the tangential ones Neumann, "
                                             "or the converse");
      }
  }
  if (!(d->mu0 > 0.0) || !(d->lambda0 >= 0.0)) return set_err(FFTM_E_INVALID, "need mu0 > 0, lambda0 >= 0");
  if (d->precision != FFTM_FP64 && d->precision != FFTM_FP32 && d->precision != FFTM_FP32_TC &&
      d->precision != FFTM_FP32_TF32)
    return set_err(FFTM_E_INVALID, "bad precision");
  if (d->precision == FFTM_FP32_TF32)
    for (int a = 0; a < 3; ++a)
      if (d->n[a] + 1 > 384)
        return set_err(FFTM_E_UNSUPPORTED, "TF32 tensor-core transforms need n <= 383 per axis");
  if (d->precision == FFTM_FP32_TC)
    for (int a = 0; a < 3; ++a)
      if (d->n[a] + 1 > 384) return set_err(FFTM_E_UNSUPPORTED, "tensor-core transforms need n <= 383 per axis");
  if (!(d->tol > 0.0) || d->max_iter < 1) return set_err(FFTM_E_INVALID, "need tol > 0 and max_iter >= 1");
  if (d->anderson_depth != 0 && (d->anderson_depth < 2 || d->anderson_depth > 4))
    return set_err(FFTM_E_INVALID, "anderson_depth must be 0 or 2..4");
  if (d->anderson_depth != 0 && d->anderson_period < 1) return set_err(FFTM_E_INVALID, "anderson_period >= 1");
  for (int a = 0; a < 3; ++a) {
    const bool per = d->bc[a][0][0] == FFTM_BC_PERIODIC;
    const int M = per ? d->n[a] : 2 * d->n[a];
    std::vector<int> r;
    if (!factor_radices(M, &r)) return set_err(FFTM_E_UNSUPPORTED, "grid sizes must be 2^a 3^b");
    if (M > 2048) return set_err(FFTM_E_UNSUPPORTED, "transform length above 2048");
  }
  return FFTM_OK;
}

struct Sizes {
  long long PX, comp_stride;
  size_t fields, tables, lawc, partial;
};

// what a problem allocates besides its fields and tables, counted for a caller's workspace: the
// staging buffer of host transfers (the largest field), the device-decided step's history and
// control block, the one-pass law table, the norm scalars, and the 256-byte alignment of every
// allocation
size_t step_extra_bytes(const fftm_problem_desc* d) {
  const size_t esz = d->precision == FFTM_FP64 ? 8 : 4;
  const size_t nvox = (size_t)d->n[0] * d->n[1] * d->n[2], npp = d->scheme == FFTM_TETRA2 ? 2 : 1;
  size_t nodes = 1;
  for (int a = 0; a < 3; ++a) nodes *= (size_t)(d->bc[a][0][0] == FFTM_BC_PERIODIC ? d->n[a] : d->n[a] + 1);
  const size_t scratch = std::max(3 * nodes, 10 * npp * nvox) * esz;
  const size_t hist = (size_t)(d->max_iter + 1) * (sizeof(double) + sizeof(int)) + 4 * sizeof(int);
  return scratch + hist + (size_t)d->n_phases * 36 * esz + 64 * sizeof(double) + sizeof(int) + 64 * 256;
}

Sizes sizes_of(const fftm_problem_desc* d) {
  Sizes s;
  const size_t esz = d->precision == FFTM_FP64 ? 8 : 4;
  int N[3];
  for (int a = 0; a < 3; ++a) N[a] = d->bc[a][0][0] == FFTM_BC_PERIODIC ? d->n[a] : d->n[a] + 1;
  s.PX = (N[0] + 7) / 8 * 8;
  s.comp_stride = (s.PX * N[1] * N[2] + 63) / 64 * 64;
  s.fields = (size_t)nsets(esz == 4) * 3 * s.comp_stride * esz;
  size_t t = 0;
  for (int a = 0; a < 3; ++a) {
    const int M = 2 * d->n[a] + 2;
    t += 3 * ((size_t)M * 2 + 16 + (size_t)M * 2 * esz + 16 + (size_t)(d->n[a] + 2) * 2 * esz + 16 +
              2 * ((size_t)(d->n[a] + 2) * esz + 16));
  }
  s.tables = t + 4096;
  s.lawc = (size_t)d->n_phases * LAWC * esz;
  s.partial = (size_t)(4 * 152 * 64) * 20 * sizeof(double);
  return s;
}

}  // namespace

// ======================================================================================
extern "C" {
static int ensure_scratch(fftm_problem* p, size_t bytes);
}

template <typename T>
static int set_load_field_t(fftm_problem* p, const void* u, int is_device, size_t bytes) {
  cudaStream_t s = p->ctx->stream;
  const void* from = u;
  if (!is_device) {
    int rc = ensure_scratch(p, bytes);
    if (rc) return rc;
    CU(cudaMemcpyAsync(p->scratch, u, bytes, cudaMemcpyHostToDevice, s));
    from = p->scratch;
  }
  if (!p->ustar) {
    DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->ustar), 3 * (size_t)p->comp_stride * sizeof(T)));
    CU(cudaMemsetAsync(p->ustar, 0, 3 * (size_t)p->comp_stride * sizeof(T), s));
  }
  T* dst[3];
  for (int q = 0; q < 3; ++q) dst[q] = reinterpret_cast<T*>(p->ustar) + q * p->comp_stride;
  CU(launch_pack<T>((const T* const*)dst, const_cast<T*>(reinterpret_cast<const T*>(from)), p->N[0], p->N[1],
                    p->N[2], p->sy, p->sz, 1, s));
  CU(cudaStreamSynchronize(s));
  p->launches++;
  return FFTM_OK;
}

extern "C" {

const char* fftm_last_error(void) { return g_last_error.c_str(); }
int fftm_version(void) { return 1; }

int fftm_ctx_create(fftm_ctx** out, int device, void* cuda_stream) {
  if (!out) return set_err(FFTM_E_INVALID, "null out");
  int count = 0;
  CU(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return set_err(FFTM_E_INVALID, "bad device index");
  CU(cudaSetDevice(device));
  fftm_ctx* c = new (std::nothrow) fftm_ctx;
  if (!c) return set_err(FFTM_E_NOMEM, "host allocation");
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  *out = c;
  return FFTM_OK;
}

int fftm_ctx_destroy(fftm_ctx* ctx) {
  delete ctx;
  return FFTM_OK;
}

int fftm_problem_workspace_bytes(const fftm_problem_desc* desc0, size_t* bytes) {
  fftm_problem_desc dres;
  int rc = resolved_desc(desc0, &dres);
  if (rc) return rc;
  const fftm_problem_desc* desc = &dres;
  rc = validate(desc);
  if (rc) return rc;
  if (!bytes) return set_err(FFTM_E_INVALID, "null bytes");
  Sizes s = sizes_of(desc);
  const long long nvox = (long long)desc->n[0] * desc->n[1] * desc->n[2];
  const size_t esz = desc->precision == FFTM_FP64 ? 8 : 4;
  const size_t vsb = (size_t)(desc->scheme == FFTM_TETRA2 ? 2 : 1) * 9 * nvox * esz;
  size_t stb = 0;  // committed state and next state; J2 also u^f and D at the commit
  for (int i = 0; i < desc->n_phases; ++i)
    if (desc->materials[i].law == FFTM_LAW_J2_LINHARD)
      stb = 2 * (size_t)(desc->scheme == FFTM_TETRA2 ? 2 : 1) * 7 * nvox * esz + (esz == 4 ? 9 : 6) * s.comp_stride * esz;
    else if (desc->materials[i].law == FFTM_LAW_CP_FCC)
      stb = 2 * (size_t)(desc->scheme == FFTM_TETRA2 ? 2 : 1) * 10 * nvox * esz;
    else if (desc->materials[i].law == FFTM_LAW_LOG_J2)
      stb = 2 * (size_t)(desc->scheme == FFTM_TETRA2 ? 2 : 1) * 7 * nvox * esz;
  const size_t c0b = desc->green == FFTM_GREEN_C0 ? 2 * (size_t)(desc->n[0] + desc->n[1] + desc->n[2] + 3) * esz : 0;
  size_t tcb = 0;  // tensor-core transform matrices: forward and inverse per component and axis
  if (desc->precision == FFTM_FP32_TC || desc->precision == FFTM_FP32_TF32)
    for (int a = 0; a < 3; ++a) {
      const size_t Kp = (size_t)(desc->n[a] + 4 + 31) / 32 * 32, R = (Kp + 127) / 128 * 128;
      tcb += 3 * 2 * R * Kp * (desc->precision == FFTM_FP32_TC ? 2 : 4);
    }
  *bytes = s.fields + s.tables + s.lawc + s.partial + vsb + stb + c0b + nvox * sizeof(uint16_t) +
           desc->n_phases * sizeof(int) + step_extra_bytes(desc) + tcb;
  return FFTM_OK;
}

int fftm_problem_destroy(fftm_problem* p) {
  if (!p) return FFTM_OK;
  if (p->ctx) cudaSetDevice(p->ctx->device);
  dev_free(p, p->fields);
  dev_free(p, p->Dbuf);
  dev_free(p, p->tables);
  dev_free(p, p->phase);
  dev_free(p, p->law_id);
  dev_free(p, p->law_c);
  dev_free(p, p->law_m);
  dev_free(p, p->partial);
  dev_free(p, p->dscal);
  dev_free(p, p->dint);
  dev_free(p, p->dctl);
  dev_free(p, p->derr);
  dev_free(p, p->scratch);
  dev_free(p, p->vs);
  dev_free(p, p->vs_test);
  dev_free(p, p->state);
  dev_free(p, p->state_next);
  dev_free(p, p->un);
  dev_free(p, p->Dn);
  dev_free(p, p->tcmat);
  dev_free(p, p->tc_err);
  dev_free(p, p->c0tab);
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < 2; ++f) {
      dev_free(p, p->tface[a][f]);
      dev_free(p, p->tface_n[a][f]);
    }
  dev_free(p, p->ustar);
  dev_free(p, p->ustar_n);
  if (p->hpin) cudaFreeHost(p->hpin);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  delete p;
  return FFTM_OK;
}

static int problem_create(fftm_ctx* ctx, const fftm_problem_desc* desc, void* workspace, size_t ws_bytes,
                          fftm_problem** out);

int fftm_problem_create(fftm_ctx* ctx, const fftm_problem_desc* desc, fftm_problem** out) {
  return problem_create(ctx, desc, nullptr, 0, out);
}

int fftm_problem_create_in(fftm_ctx* ctx, const fftm_problem_desc* desc, void* workspace, size_t bytes,
                           fftm_problem** out) {
  if (!workspace) return set_err(FFTM_E_INVALID, "null workspace");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return set_err(FFTM_E_INVALID, "workspace must be 256-byte aligned");
  size_t need = 0;
  int rc = fftm_problem_workspace_bytes(desc, &need);
  if (rc) return rc;
  if (bytes < need) return set_err(FFTM_E_NOMEM, "workspace smaller than fftm_problem_workspace_bytes");
  return problem_create(ctx, desc, workspace, bytes, out);
}

static int problem_create(fftm_ctx* ctx, const fftm_problem_desc* desc0, void* workspace, size_t ws_bytes,
                          fftm_problem** out) {
  if (!ctx || !out) return set_err(FFTM_E_INVALID, "null ctx or out");
  fftm_problem_desc dres;
  int rc = resolved_desc(desc0, &dres);
  if (rc) return rc;
  const fftm_problem_desc* desc = &dres;
  rc = validate(desc);
  if (rc) return rc;
  CU(cudaSetDevice(ctx->device));
  std::unique_ptr<fftm_problem> p(new (std::nothrow) fftm_problem);
  if (!p) return set_err(FFTM_E_NOMEM, "host allocation");
  p->arena = static_cast<char*>(workspace);
  p->arena_size = workspace ? ws_bytes : 0;
  p->ctx = ctx;
  p->desc = *desc;
  p->mats.assign(desc->materials, desc->materials + desc->n_phases);
  p->desc.materials = nullptr;
  p->desc.phase = nullptr;
  p->prec = desc->precision;
  p->esz = desc->precision == FFTM_FP64 ? 8 : 4;
  p->tetra = desc->scheme == FFTM_TETRA2;
  std::memset(&p->load, 0, sizeof(p->load));
  std::memset(&p->load_n, 0, sizeof(p->load_n));
  p->committed = 0;
  for (int a = 0; a < 3; ++a) {
    p->n[a] = desc->n[a];
    p->h[a] = desc->h[a];
    p->periodic[a] = desc->bc[a][0][0] == FFTM_BC_PERIODIC;
    p->N[a] = p->periodic[a] ? p->n[a] : p->n[a] + 1;
  }
  Sizes sz = sizes_of(desc);
  p->PX = sz.PX;
  p->sy = sz.PX;
  p->sz = sz.PX * p->N[1];
  p->comp_stride = sz.comp_stride;
  p->nvox = (long long)p->n[0] * p->n[1] * p->n[2];
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) {
      const int sl = face_sym(desc->bc[a][0][q]), sr = face_sym(desc->bc[a][1][q]);
      p->sgn[q][a][0] = p->periodic[a] ? 1 : sl;
      p->sgn[q][a][1] = p->periodic[a] ? 1 : sr;
      p->kind[q][a] = kind_of(sl, sr, p->periodic[a]);
      int lo, L;
      kind_range(p->kind[q][a], p->n[a], &lo, &L);
      p->lo[q][a] = lo;
      p->hi[q][a] = lo + L;
      p->plans[q][a] = make_plan(p->kind[q][a], p->n[a]);
    }
  for (int a = 0; a < 3; ++a) {
    p->maxM[a] = 0;
    p->maxL[a] = 0;
    for (int q = 0; q < 3; ++q) {
      p->maxM[a] = std::max(p->maxM[a], p->plans[q][a].M);
      p->maxL[a] = std::max(p->maxL[a], p->plans[q][a].L);
    }
  }
  // ---- device allocations ----
  const cudaStream_t s = ctx->stream;
  if (dev_alloc(p.get(), reinterpret_cast<void**>(&p->fields), sz.fields) != cudaSuccess) {
    cudaGetLastError();
    return set_err(FFTM_E_NOMEM, "device allocation of the fields failed");
  }
  CU(cudaMemsetAsync(p->fields, 0, sz.fields, s));
  bool has_j2 = false, has_cp = false, has_lj2 = false, finite = false;
  for (int i = 0; i < desc->n_phases; ++i) {
    const int law = desc->materials[i].law;
    const bool fin = law == FFTM_LAW_SVK_CUBIC || law == FFTM_LAW_NEO_HOOKE || law == FFTM_LAW_CP_FCC ||
                     law == FFTM_LAW_LOG_J2;
    if (law == FFTM_LAW_B0_LINEAR || fin) p->sym = 0;
    has_j2 |= law == FFTM_LAW_J2_LINHARD;
    has_cp |= law == FFTM_LAW_CP_FCC;
    has_lj2 |= law == FFTM_LAW_LOG_J2;
    finite |= fin;
  }
  p->nst = has_cp ? 10 : ((has_j2 || has_lj2) ? 7 : 0);
  p->slaw = has_cp ? 2 : (has_j2 ? 1 : (has_lj2 ? 4 : 0));
  p->inc_ok = has_j2 && !finite;
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->vs), (size_t)(p->tetra ? 2 : 1) * (p->sym ? 6 : 9) * p->nvox * p->esz));
  if (p->nst) {
    const size_t sb = (size_t)(p->tetra ? 2 : 1) * p->nst * p->nvox * p->esz;
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->state), sb));
    CU(cudaMemsetAsync(p->state, 0, sb, s));  // J2: e = 0, p = 0; crystal plasticity: F^p - 1 = 0, Gamma = 0
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->state_next), sb));
    CU(cudaMemsetAsync(p->state_next, 0, sb, s));
  }
  if (p->inc_ok) {
    {
      const size_t ub = (size_t)(p->esz == 4 ? 6 : 3) * p->comp_stride * p->esz;
      DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->un), ub));
      CU(cudaMemsetAsync(p->un, 0, ub, s));
      DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->Dn), 3 * p->comp_stride * p->esz));
      CU(cudaMemsetAsync(p->Dn, 0, 3 * p->comp_stride * p->esz, s));
    }
  }
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->phase), p->nvox * sizeof(uint16_t)));
  CU(cudaMemcpyAsync(p->phase, desc->phase, p->nvox * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->partial), sz.partial));
  p->partial_len = sz.partial / sizeof(double);
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->dscal), 64 * sizeof(double)));
  CU(cudaMemsetAsync(p->dscal, 0, 64 * sizeof(double), s));
  CU(cudaMallocHost(&p->hpin, 64 * sizeof(double)));
  // ---- tables: plans and Green half-angle tables ----
  std::vector<unsigned char> tab;
  auto put = [&](const void* src, size_t bytes) {
    size_t off = (tab.size() + 15) & ~(size_t)15;
    tab.resize(off + bytes);
    std::memcpy(tab.data() + off, src, bytes);
    return off;
  };
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) {
      const HostPlan& h = p->plans[q][a];
      p->off_perm[q][a] = put(h.perm.data(), h.perm.size() * sizeof(int16_t));
      std::vector<double> s2(h.L), c2(h.L);
      for (int k = 0; k < h.L; ++k) {
        bool z, pi;
        const double xi = kind_xi(h.kind, h.n, k, &z, &pi);
        const double sv = z ? 0.0 : std::sin(0.5 * xi);
        const double cv = pi ? 0.0 : std::cos(0.5 * xi);
        s2[k] = sv * sv;
        c2[k] = cv * cv;
      }
      if (p->esz == 8) {
        p->off_tw[q][a] = put(h.tw.data(), h.tw.size() * 8);
        p->off_qw[q][a] = put(h.qw.data(), h.qw.size() * 8);
        p->off_S2[q][a] = put(s2.data(), s2.size() * 8);
        p->off_C2[q][a] = put(c2.data(), c2.size() * 8);
      } else {
        std::vector<float> tw(h.tw.begin(), h.tw.end()), qw(h.qw.begin(), h.qw.end());
        std::vector<float> s2f(s2.begin(), s2.end()), c2f(c2.begin(), c2.end());
        p->off_tw[q][a] = put(tw.data(), tw.size() * 4);
        p->off_qw[q][a] = put(qw.data(), qw.size() * 4);
        p->off_S2[q][a] = put(s2f.data(), s2f.size() * 4);
        p->off_C2[q][a] = put(c2f.data(), c2f.size() * 4);
      }
    }
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->tables), tab.size()));
  CU(cudaMemcpy(p->tables, tab.data(), tab.size(), cudaMemcpyHostToDevice));
  if (desc->precision == FFTM_FP32_TC) {
    p->tc = 1;
    std::vector<uint16_t> mats;
    // R x Kp zero-padded (R = Kp, on the x axis Kp rounded up to 128), in 32-column chunks
    // laid out as the shared-memory core matrices the tensor cores read: element (m, jj) of
    // chunk c at c R 32 + (m>>3) 256 + (jj>>3) 64 + (m&7) 8 + (jj&7) (BF16 elements).
    // On the x axis the tensor-core pass indexes its input and output by x - xb, xb = lo
    // rounded down to a multiple of 4 (aligned row copies), so there the rows and columns
    // are shifted by lo - xb.
    auto put_mat = [&](const std::vector<double>& M, int L, int Kp, int R, int sh) {
      size_t off = (mats.size() + 63) & ~(size_t)63;  // 128-byte aligned
      mats.resize(off + (size_t)R * Kp, 0);
      for (int r0 = 0; r0 < L; ++r0)
        for (int c0 = 0; c0 < L; ++c0) {
          const int m = r0 + sh, c = c0 + sh;
          const int ch = c / 32, jj = c % 32;
          const size_t at = (size_t)ch * R * 32 + (size_t)(m >> 3) * 256 + (jj >> 3) * 64 + (m & 7) * 8 + (jj & 7);
          mats[off + at] = to_bf16(M[(size_t)r0 * L + c0]);
        }
      return off * sizeof(uint16_t);
    };
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 3; ++a) {
        std::vector<double> F, I;
        int L;
        dense_forward(p->kind[q][a], p->n[a], &F, &L);
        dense_inverse(p->kind[q][a], p->n[a], &I);
        const int col0 = a == 0 ? (p->plans[q][a].lo & 3) : 0;
        const int Kp = (L + col0 + 31) / 32 * 32;
        // shared memory of one CTA (two pencil tiles, at least two matrix chunks) and TMEM:
        // Kp up to 288 on the x axis, 352 on y and z
        if (!pass_tc_fits(Kp, a))
          return set_err(FFTM_E_UNSUPPORTED, "tensor-core transforms need lengths up to 288 (x) and 352 (y, z)");
        p->tcKp[q][a] = Kp;
        const int R = pass_tc_rows(Kp, a);
        p->off_tcf[q][a] = put_mat(F, L, Kp, R, col0);
        p->off_tci[q][a] = put_mat(I, L, Kp, R, col0);
      }
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->tcmat), mats.size() * sizeof(uint16_t)));
    CU(cudaMemcpy(p->tcmat, mats.data(), mats.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->tc_err), sizeof(int)));
    CU(cudaMemset(p->tc_err, 0, sizeof(int)));
  }
  if (desc->precision == FFTM_FP32_TF32) {
    p->tf = 1;
    std::vector<float> mats;
    // R x Kp zero-padded (R = Kp, on the x axis Kp rounded up to 128), in 32-column chunks in
    // the K-major core-matrix order of FP32 elements: element (m, jj) of chunk c at
    // c R 32 + (m>>3) 256 + (jj>>2) 32 + (m&7) 4 + (jj&3).  On the x axis rows and columns are
    // shifted by lo - xb, xb = lo rounded down to a multiple of 4 (aligned 16-byte copies).
    auto put_mat = [&](const std::vector<double>& M, int L, int Kp, int R, int sh) {
      size_t off = (mats.size() + 31) & ~(size_t)31;  // 128-byte aligned
      mats.resize(off + (size_t)R * Kp, 0.f);
      for (int r0 = 0; r0 < L; ++r0)
        for (int c0 = 0; c0 < L; ++c0) {
          const int m = r0 + sh, c = c0 + sh;
          if (m >= R) continue;  // output 256 of a 257-output y / z transform: its own row
          const int ch = c / 32, jj = c % 32;
          const size_t at = (size_t)ch * R * 32 + (size_t)(m >> 3) * 256 + (jj >> 2) * 32 + (m & 7) * 4 + (jj & 3);
          mats[off + at] = to_tf32(M[(size_t)r0 * L + c0]);
        }
      return off * sizeof(float);
    };
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 3; ++a) {
        std::vector<double> F, I;
        int L;
        dense_forward(p->kind[q][a], p->n[a], &F, &L);
        dense_inverse(p->kind[q][a], p->n[a], &I);
        const int col0 = a == 0 ? (p->plans[q][a].lo & 3) : 0;
        const int Kp = (L + col0 + 31) / 32 * 32;
        // y, z with 257 outputs (DCT-I over 256 intervals): 256 on the tensor cores, so that two
        // accumulators fit TMEM, and output 256 as an FP32 dot product in the producers
        const bool xt = a != 0 && L == 257 && pass_tf32_fits(256, a, 1);
        const int Kn = xt ? 256 : Kp;
        if (!pass_tf32_fits(Kn, a, xt ? 1 : 0))
          return set_err(FFTM_E_UNSUPPORTED, "TF32 tensor-core transforms need lengths up to 384 per axis");
        p->tcKp[q][a] = Kp;
        p->tcKn[q][a] = Kn;
        p->tcx[q][a] = xt ? 1 : 0;
        const int R = pass_tf32_rows(Kn, a);
        p->off_tcf[q][a] = put_mat(F, L, Kp, R, col0);
        p->off_tci[q][a] = put_mat(I, L, Kp, R, col0);
        if (xt) {  // row 256 over the K positions, FP32, zero-padded to Kp
          for (int inv = 0; inv < 2; ++inv) {
            const std::vector<double>& M = inv ? I : F;
            const size_t off = (mats.size() + 31) & ~(size_t)31;
            mats.resize(off + (size_t)Kp, 0.f);
            for (int c0 = 0; c0 < L; ++c0) mats[off + c0] = (float)M[(size_t)256 * L + c0];
            (inv ? p->off_tcxi : p->off_tcxf)[q][a] = off * sizeof(float);
          }
        }
      }
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->tcmat), mats.size() * sizeof(float)));
    CU(cudaMemcpy(p->tcmat, mats.data(), mats.size() * sizeof(float), cudaMemcpyHostToDevice));
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->tc_err), sizeof(int)));
    CU(cudaMemset(p->tc_err, 0, sizeof(int)));
  }
  // ---- law tables ----
  std::vector<int> lid(desc->n_phases);
  std::vector<double> lc((size_t)desc->n_phases * LAWC, 0.0);
  for (int i = 0; i < desc->n_phases; ++i) {
    const fftm_material& m = desc->materials[i];
    lid[i] = m.law;
    double* c = &lc[(size_t)i * LAWC];
    if (m.law == FFTM_LAW_CUBIC_ELASTIC || m.law == FFTM_LAW_SVK_CUBIC) {
      double R[3][3], Cm[6][6];
      quat_rot(m.quat, R);
      cubic_mandel(m.params[0], m.params[1], m.params[2], R, Cm);
      int k = 0;
      for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) c[k++] = Cm[a][b];
    } else if (m.law == FFTM_LAW_J2_LINHARD) {
      for (int k = 0; k < 4; ++k) c[k] = m.params[k];
    } else if (m.law == FFTM_LAW_LOG_J2) {
      for (int k = 0; k < 3; ++k) c[k] = m.params[k];
    } else if (m.law == FFTM_LAW_CP_FCC) {
      double R[3][3], Cm[6][6];
      quat_rot(m.quat, R);
      cubic_mandel(m.params[0], m.params[1], m.params[2], R, Cm);
      int k = 0;
      for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) c[k++] = Cm[a][b];
      for (int j = 0; j < 6; ++j) c[21 + j] = m.params[3 + j];  // gdot0, n, tau0, tau_inf, h0, dt
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c[27 + 3 * a + b] = R[a][b];
    } else {
      c[0] = m.params[0];
      c[1] = m.params[1];
    }
  }
  // the small-strain elastic phases' Mandel stiffness for the one-pass residual: float4 k = 3 bp + rp
  // holds (C[2rp][2bp], C[2rp+1][2bp], C[2rp][2bp+1], C[2rp+1][2bp+1]) (isotropic: lambda 1 (x) 1 + 2 mu I)
  std::vector<double> lm((size_t)desc->n_phases * 36, 0.0);
  for (int i = 0; i < desc->n_phases; ++i) {
    const fftm_material& m = desc->materials[i];
    double Cm[6][6] = {};
    if (m.law == FFTM_LAW_CUBIC_ELASTIC) {
      double R[3][3];
      quat_rot(m.quat, R);
      cubic_mandel(m.params[0], m.params[1], m.params[2], R, Cm);
    } else if (m.law == FFTM_LAW_ISO_ELASTIC) {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Cm[a][b] = m.params[0];
      for (int a = 0; a < 6; ++a) Cm[a][a] += 2.0 * m.params[1];
    }
    double* c = &lm[(size_t)i * 36];
    for (int bp = 0; bp < 3; ++bp)
      for (int rp = 0; rp < 3; ++rp) {
        double* f = c + 4 * (3 * bp + rp);
        f[0] = Cm[2 * rp][2 * bp];
        f[1] = Cm[2 * rp + 1][2 * bp];
        f[2] = Cm[2 * rp][2 * bp + 1];
        f[3] = Cm[2 * rp + 1][2 * bp + 1];
      }
  }
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->law_m), lm.size() * p->esz));
  if (p->esz == 8) {
    CU(cudaMemcpy(p->law_m, lm.data(), lm.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> lf(lm.begin(), lm.end());
    CU(cudaMemcpy(p->law_m, lf.data(), lf.size() * 4, cudaMemcpyHostToDevice));
  }
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->law_id), lid.size() * sizeof(int)));
  CU(cudaMemcpy(p->law_id, lid.data(), lid.size() * sizeof(int), cudaMemcpyHostToDevice));
  DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->law_c), lc.size() * p->esz));
  if (p->esz == 8) {
    CU(cudaMemcpy(p->law_c, lc.data(), lc.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> lf(lc.begin(), lc.end());
    CU(cudaMemcpy(p->law_c, lf.data(), lf.size() * 4, cudaMemcpyHostToDevice));
  }
  if (desc->green == FFTM_GREEN_C0) {
    // sin and cos of xi / 2 at the node positions m = 0 .. n of each axis (xi = pi m / n, the
    // DCT-I / DST-I frequency of position m), with the exact zeros sin = 0 at m = 0 and cos = 0
    // at m = n (the null rule is decided on them)
    p->c0 = 1;
    std::vector<double> t;
    for (int a = 0; a < 3; ++a) {
      const int n = p->n[a];
      for (int m = 0; m < p->N[a]; ++m) t.push_back(m == 0 ? 0.0 : std::sin(0.5 * kPi * m / n));
      for (int m = 0; m < p->N[a]; ++m) t.push_back(m == n ? 0.0 : std::cos(0.5 * kPi * m / n));
    }
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->c0tab), t.size() * p->esz));
    if (p->esz == 8) {
      CU(cudaMemcpy(p->c0tab, t.data(), t.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> tf(t.begin(), t.end());
      CU(cudaMemcpy(p->c0tab, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice));
    }
  }
  if (p->arena) {  // everything the solve allocates later comes from the workspace now
    const size_t nodes3 = (size_t)3 * p->N[0] * p->N[1] * p->N[2];
    const size_t pts10 = (size_t)10 * (p->tetra ? 2 : 1) * (size_t)p->nvox;
    int rc2 = ensure_scratch(p.get(), (nodes3 > pts10 ? nodes3 : pts10) * p->esz);
    if (rc2) return rc2;
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->derr), (desc->max_iter + 1) * sizeof(double)));
    p->derr_len = desc->max_iter + 1;
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->dint), (desc->max_iter + 1) * sizeof(int)));
    p->dint_len = desc->max_iter + 1;
    DEVALLOC(dev_alloc(p.get(), reinterpret_cast<void**>(&p->dctl), 4 * sizeof(int)));
  }
  CU(cudaStreamSynchronize(s));
  *out = p.release();
  return FFTM_OK;
}

int fftm_set_phase(fftm_problem* p, const uint16_t* phase) {
  if (!p || !phase) return set_err(FFTM_E_INVALID, "null argument");
  CU(cudaSetDevice(p->ctx->device));
  CU(cudaMemcpyAsync(p->phase, phase, p->nvox * sizeof(uint16_t), cudaMemcpyHostToDevice, p->ctx->stream));
  CU(cudaStreamSynchronize(p->ctx->stream));
  return FFTM_OK;
}

int fftm_set_load(fftm_problem* p, const fftm_load* load) {
  if (!p || !load) return set_err(FFTM_E_INVALID, "null argument");
  for (int a = 0; a < 3; ++a)
    if (p->periodic[a])
      for (int q = 0; q < 3; ++q)
        if (load->A[q][a] != 0.0) return set_err(FFTM_E_INVALID, "u* depends on a periodic coordinate");
  // quadratic monomials x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2 and the axes they contain
  static const int mono_axes[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < 6; ++k)
      if (load->Q[q][k] != 0.0 && (p->periodic[mono_axes[k][0]] || p->periodic[mono_axes[k][1]]))
        return set_err(FFTM_E_INVALID, "u* depends on a periodic coordinate");
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < 2; ++f)
      for (int q = 0; q < 3; ++q)
        if (load->T[a][f][q] != 0.0 && p->desc.bc[a][f][q] != FFTM_BC_NEUMANN)
          return set_err(FFTM_E_INVALID, "a traction on a face where that component is not Neumann");
  fftm_load ld = *load;
  if (ld.mixed) {
    if (ld.mixed & ~0x3F) return set_err(FFTM_E_INVALID, "mixed mask has bits beyond the six strain components");
    if (!p->sym) return set_err(FFTM_E_INVALID, "normal-mixed loading needs small-strain laws (symmetric stress)");
    for (int k = 0; k < 6; ++k)
      if (((ld.mixed >> k) & 1) && (p->periodic[kVoigt[k][0]] || p->periodic[kVoigt[k][1]]))
        return set_err(FFTM_E_INVALID, "a free strain component of a mixed load lies along a periodic axis");
    if (ld.mixed == p->mixed_prev)  // free components start where the previous mixed step ended
      for (int k = 0; k < 6; ++k)
        if ((ld.mixed >> k) & 1) {
          const int i = kVoigt[k][0], j = kVoigt[k][1];
          ld.A[i][j] = p->mixed_A[i][j];
          ld.A[j][i] = p->mixed_A[j][i];
        }
  }
  p->load = ld;
  return FFTM_OK;
}

int fftm_host_dense_transform(int kind, int n, int inverse, double* out, int* L_out) {
  if (kind < K_DFT || kind > K_DST3 || n < 2 || n > 4096 || (inverse != 0 && inverse != 1) || !L_out)
    return set_err(FFTM_E_INVALID, "bad transform kind, length or output");
  std::vector<double> M;
  int L = 0;
  if (inverse) {
    int lo;
    kind_range(kind, n, &lo, &L);
    if (out) dense_inverse(kind, n, &M);
  } else if (out) {
    dense_forward(kind, n, &M, &L);
  } else {
    int lo;
    kind_range(kind, n, &lo, &L);
  }
  *L_out = L;
  if (out) std::memcpy(out, M.data(), M.size() * sizeof(double));
  return FFTM_OK;
}

int fftm_dt1d(int device, int kind, int n, int inverse, const double* in, double* out) {
  if (kind < K_DFT || kind > K_DST3 || n < 2 || n > 4096 || (inverse != 0 && inverse != 1) || !in || !out)
    return set_err(FFTM_E_INVALID, "bad transform kind, length or array");
  int lo = 0, L = 0;
  kind_range(kind, n, &lo, &L);
  // an n x 2 x 2 problem, periodic along y and z, the kind's face pair on x for every component
  static const int pair[5][2] = {{FFTM_BC_PERIODIC, FFTM_BC_PERIODIC}, {FFTM_BC_NEUMANN, FFTM_BC_NEUMANN},
                                 {FFTM_BC_NEUMANN, FFTM_BC_DIRICHLET}, {FFTM_BC_DIRICHLET, FFTM_BC_DIRICHLET},
                                 {FFTM_BC_DIRICHLET, FFTM_BC_NEUMANN}};
  std::vector<uint16_t> phase((size_t)n * 4, 0);
  fftm_material mat;
  std::memset(&mat, 0, sizeof(mat));
  mat.law = FFTM_LAW_ISO_ELASTIC;
  mat.params[0] = 1.0;
  mat.params[1] = 1.0;
  mat.quat[0] = 1.0;
  fftm_problem_desc d;
  std::memset(&d, 0, sizeof(d));
  d.n[0] = n;
  d.n[1] = d.n[2] = 2;
  d.h[0] = d.h[1] = d.h[2] = 1.0;
  d.phase = phase.data();
  d.n_phases = 1;
  d.materials = &mat;
  for (int f = 0; f < 2; ++f)
    for (int q = 0; q < 3; ++q) {
      d.bc[0][f][q] = pair[kind][f];
      d.bc[1][f][q] = d.bc[2][f][q] = FFTM_BC_PERIODIC;
    }
  d.scheme = FFTM_HEX1;
  d.green = FFTM_GREEN_B0;
  d.lambda0 = d.mu0 = 1.0;
  d.precision = FFTM_FP64;
  d.tol = 1.0;
  d.max_iter = 1;
  d.anderson_depth = 0;
  d.anderson_period = 3;
  fftm_ctx* ctx = nullptr;
  int rc = fftm_ctx_create(&ctx, device, nullptr);
  if (rc) return rc;
  fftm_problem* p = nullptr;
  rc = fftm_problem_create(ctx, &d, &p);
  if (rc) {
    fftm_ctx_destroy(ctx);
    return rc;
  }
  // component 0: forward, the input on all four (y, z) lines (the y and z DFTs of a constant
  // put 4 x the x transform on line (0, 0)); inverse, 4 x the input on line (0, 0) alone (the
  // normalised y and z inverses spread it to every line)
  const int N0 = p->N[0];
  const size_t line = (size_t)N0, count = 3 * 4 * line;
  std::vector<double> f(count, 0.0);
  for (int l = 0; l < (inverse ? 1 : 4); ++l)
    for (int c = 0; c < L; ++c) f[l * line + lo + c] = inverse ? 4.0 * in[c] : in[c];
  rc = fftm_set_field(p, FFTM_FIELD_WORK, f.data(), 0, count * sizeof(double));
  if (!rc) rc = fftm_apply(p, inverse ? FFTM_OP_DT_INVERSE : FFTM_OP_DT_FORWARD, nullptr);
  if (!rc) rc = fftm_get_field(p, FFTM_FIELD_WORK, f.data(), 0, count * sizeof(double));
  if (!rc)
    for (int c = 0; c < L; ++c) out[c] = inverse ? f[lo + c] : 0.25 * f[lo + c];
  fftm_problem_destroy(p);
  fftm_ctx_destroy(ctx);
  return rc;
}

int fftm_host_reference_medium(const fftm_problem_desc* d, double* lambda0, double* mu0) {
  if (!d || !lambda0 || !mu0) return set_err(FFTM_E_INVALID, "null argument");
  double l0 = d->lambda0, m0 = d->mu0;
  if (l0 == FFTM_REF_AUTO || m0 == FFTM_REF_AUTO) {
    if (!d->materials || d->n_phases < 1) return set_err(FFTM_E_INVALID, "FFTM_REF_AUTO needs the materials");
    double lmin = 0.0, lmax = 0.0, mmin = 0.0, mmax = 0.0;
    for (int i = 0; i < d->n_phases; ++i) {
      double l, m;
      phase_lame(d->materials[i], &l, &m);
      lmin = (i == 0 || l < lmin) ? l : lmin;
      lmax = (i == 0 || l > lmax) ? l : lmax;
      mmin = (i == 0 || m < mmin) ? m : mmin;
      mmax = (i == 0 || m > mmax) ? m : mmax;
    }
    if (l0 == FFTM_REF_AUTO) l0 = 0.5 * (lmin + lmax);
    if (m0 == FFTM_REF_AUTO) m0 = 0.5 * (mmin + mmax);
  }
  *lambda0 = l0;
  *mu0 = m0;
  return FFTM_OK;
}

int fftm_host_mixed_increment(const double* sig, int mask, double lambda0, double mu0, double* d_out) {
  if (!sig || !d_out || (mask & ~0x3F) || !(mu0 > 0.0) || !(lambda0 >= 0.0))
    return set_err(FFTM_E_INVALID, "bad mixed increment arguments");
  double s3[3][3], d[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s3[i][j] = sig[i * 3 + j];
  mixed_increment(s3, mask, lambda0, mu0, d);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) d_out[i * 3 + j] = d[i][j];
  return FFTM_OK;
}

int fftm_set_load_field(fftm_problem* p, const void* ustar, int is_device, size_t bytes) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  CU(cudaSetDevice(p->ctx->device));
  if (!ustar) {
    CU(cudaStreamSynchronize(p->ctx->stream));
    dev_free(p, p->ustar);
    p->ustar = nullptr;
    return FFTM_OK;
  }
  if (p->load.mixed) return set_err(FFTM_E_INVALID, "a u* field with a normal-mixed load");
  const size_t need = 3 * (size_t)p->N[0] * p->N[1] * p->N[2] * p->esz;
  if (bytes != need) return set_err(FFTM_E_INVALID, "byte count does not match the node field");
  if (p->esz == 8) return set_load_field_t<double>(p, ustar, is_device, bytes);
  return set_load_field_t<float>(p, ustar, is_device, bytes);
}

int fftm_set_face_traction(fftm_problem* p, int axis, int face, const void* t, int t_is_device, size_t bytes) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  if (axis < 0 || axis > 2 || face < 0 || face > 1) return set_err(FFTM_E_INVALID, "bad axis or face");
  if (p->periodic[axis]) return set_err(FFTM_E_INVALID, "a periodic axis has no faces to load");
  CU(cudaSetDevice(p->ctx->device));
  const int nb = p->n[axis == 0 ? 1 : 0], nc = p->n[axis == 2 ? 1 : 2];
  const size_t cnt = (size_t)3 * nb * nc, need = cnt * p->esz;
  if (!t) {
    CU(cudaStreamSynchronize(p->ctx->stream));
    dev_free(p, p->tface[axis][face]);
    p->tface[axis][face] = nullptr;
    return FFTM_OK;
  }
  if (bytes != need) return set_err(FFTM_E_INVALID, "byte count does not match 3 x the face's voxels");
  std::vector<unsigned char> h(need);
  if (t_is_device) {
    CU(cudaMemcpy(h.data(), t, need, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h.data(), t, need);
  }
  for (int q = 0; q < 3; ++q) {
    if (p->desc.bc[axis][face][q] == FFTM_BC_NEUMANN) continue;
    for (size_t k = 0; k < (size_t)nb * nc; ++k) {
      const double v = p->esz == 8 ? reinterpret_cast<const double*>(h.data())[q * (size_t)nb * nc + k]
                                   : reinterpret_cast<const float*>(h.data())[q * (size_t)nb * nc + k];
      if (v != 0.0) return set_err(FFTM_E_INVALID, "a traction on a face where that component is not Neumann");
    }
  }
  CU(cudaStreamSynchronize(p->ctx->stream));
  if (!p->tface[axis][face]) DEVALLOC(dev_alloc(p, reinterpret_cast<void**>(&p->tface[axis][face]), need));
  CU(cudaMemcpy(p->tface[axis][face], h.data(), need, cudaMemcpyHostToDevice));
  return FFTM_OK;
}

int fftm_get_load(const fftm_problem* p, fftm_load* out) {
  if (!p || !out) return set_err(FFTM_E_INVALID, "null argument");
  *out = p->load;
  return FFTM_OK;
}

int fftm_solve_step(fftm_problem* p, fftm_step_report* report, double* err_history, int* accel_history,
                    int history_len) {
  if (!p || !report) return set_err(FFTM_E_INVALID, "null argument");
  CU(cudaSetDevice(p->ctx->device));
  if (p->esz == 8) return solve_step_t<double>(p, report, err_history, accel_history, history_len);
  return solve_step_t<float>(p, report, err_history, accel_history, history_len);
}

int fftm_field_bytes(const fftm_problem* p, int field, size_t* bytes) {
  if (!p || !bytes) return set_err(FFTM_E_INVALID, "null argument");
  const size_t nodes = (size_t)p->N[0] * p->N[1] * p->N[2];
  const size_t npp = p->tetra ? 2 : 1;
  switch (field) {
    case FFTM_FIELD_U:
    case FFTM_FIELD_U_LO:
    case FFTM_FIELD_WORK:
    case FFTM_FIELD_D: *bytes = 3 * nodes * p->esz; return FFTM_OK;
    case FFTM_FIELD_GRAD: *bytes = 9 * npp * p->nvox * p->esz; return FFTM_OK;
    case FFTM_FIELD_STRESS: *bytes = (p->sym ? 6 : 9) * npp * p->nvox * p->esz; return FFTM_OK;
    case FFTM_FIELD_STATE:
      if (!p->state) return set_err(FFTM_E_INVALID, "the problem has no phase with internal variables");
      *bytes = (size_t)p->nst * npp * p->nvox * p->esz;
      return FFTM_OK;
    default: return set_err(FFTM_E_INVALID, "unknown field");
  }
}

int fftm_set_option(fftm_problem* p, int option, int value) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  switch (option) {
    case FFTM_OPT_RESIDUAL_PASSES:
      if (value < 0 || value > 2) return set_err(FFTM_E_INVALID, "residual passes: 0 (tuned), 1 or 2");
      p->res_passes = value;
      p->res_two_pass = value == 0 ? -1 : (value == 2 ? 1 : 0);
      if (value == 1 && p->res_tile == 0) p->res_two_pass = -1;  // the tile height is still tuned
      return FFTM_OK;
    case FFTM_OPT_DEVICE_LOOP:
      if (value != 0 && value != 1) return set_err(FFTM_E_INVALID, "device loop: 0 or 1");
      p->dev_loop = value;
      return FFTM_OK;
    case FFTM_OPT_CUDA_GRAPH:
      if (value != 0 && value != 1) return set_err(FFTM_E_INVALID, "CUDA graph: 0 or 1");
      p->graph = value;
      return FFTM_OK;
    case FFTM_OPT_RESIDUAL_TILE:
      if (value != 0 && value != 8 && value != 16) return set_err(FFTM_E_INVALID, "residual tile: 0 (tuned), 8 or 16");
      p->res_tile = value;
      if (value) p->res_fy = value;
      p->res_two_pass = p->res_passes == 2 ? 1 : ((p->res_passes == 1 && value) ? 0 : -1);
      return FFTM_OK;
    default: return set_err(FFTM_E_INVALID, "unknown option");
  }
}

int fftm_device_fma_rate(int device, int fp64, double* flops_per_s) {
  if (!flops_per_s) return set_err(FFTM_E_INVALID, "null output");
  int count = 0;
  CU(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return set_err(FFTM_E_INVALID, "bad device index");
  CU(cudaSetDevice(device));
  const double r = fma_peak_flops(fp64 ? 1 : 0);
  if (r <= 0.0) return set_err(FFTM_E_CUDA, "FMA probe failed");
  *flops_per_s = r;
  return FFTM_OK;
}

int fftm_tuning_table(char* buf, size_t len, size_t* needed) {
  std::string out;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : g_tune_table) out += kv.first + ": " + kv.second + "\n";
  }
  if (needed) *needed = out.size() + 1;
  if (buf && len > 0) {
    const size_t n = out.size() < len - 1 ? out.size() : len - 1;
    std::memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return FFTM_OK;
}

int fftm_problem_layout(const fftm_problem* p, int N[3], int* precision, int* device) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  if (N)
    for (int a = 0; a < 3; ++a) N[a] = p->N[a];
  if (precision) *precision = p->desc.precision;
  if (device) *device = p->ctx->device;
  return FFTM_OK;
}

static int ensure_scratch(fftm_problem* p, size_t bytes) {
  if (p->scratch_bytes >= bytes) return FFTM_OK;
  dev_free(p, p->scratch);
  p->scratch = nullptr;
  p->scratch_bytes = 0;
  if (dev_alloc(p, reinterpret_cast<void**>(&p->scratch), bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_err(FFTM_E_NOMEM, "scratch allocation failed");
  }
  p->scratch_bytes = bytes;
  return FFTM_OK;
}

}  // extern "C"

template <typename T>
static int get_field_t(fftm_problem* p, int field, void* dst, int dst_is_device, size_t bytes) {
  cudaStream_t s = p->ctx->stream;
  void* target = dst;
  if (!dst_is_device) {
    int rc = ensure_scratch(p, bytes);
    if (rc) return rc;
    target = p->scratch;
  }
  if (field == FFTM_FIELD_STATE) {
    CU(launch_state_io<T>(commit_params<T>(p), p->tetra, reinterpret_cast<T*>(target), nullptr, s));
    p->launches++;
    if (!dst_is_device) CU(cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return FFTM_OK;
  }
  if (field == FFTM_FIELD_U_LO && p->esz == 8) {  // FP64: no low part
    CU(cudaMemsetAsync(target, 0, bytes, s));
  } else if (field == FFTM_FIELD_U || field == FFTM_FIELD_U_LO || field == FFTM_FIELD_WORK || field == FFTM_FIELD_D) {
    const T* src[3];
    for (int q = 0; q < 3; ++q) {
      if (field == FFTM_FIELD_U_LO) {
        src[q] = field_ptr<T>(p, SET_UL + p->cur, q);
      } else if (field == FFTM_FIELD_D) {
        if (!p->Dbuf) return set_err(FFTM_E_INVALID, "D is written by FFTM_OP_RESIDUAL first");
        src[q] = reinterpret_cast<const T*>(p->Dbuf) + q * p->comp_stride;
      } else {
        src[q] = field_ptr<T>(p, field == FFTM_FIELD_U ? SET_UH + p->cur : SET_WORK, q);
      }
    }
    CU(launch_pack<T>(src, reinterpret_cast<T*>(target), p->N[0], p->N[1], p->N[2], p->sy, p->sz, 0, s));
  } else {
    ResParams<T> R = res_params<T>(p, p->cur, nullptr, nullptr);
    T* g = field == FFTM_FIELD_GRAD ? reinterpret_cast<T*>(target) : nullptr;
    T* st = field == FFTM_FIELD_STRESS ? reinterpret_cast<T*>(target) : nullptr;
    CU(launch_voxel_fields<T>(R, p->tetra, g, st, s));
  }
  p->launches++;
  if (!dst_is_device) CU(cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return FFTM_OK;
}

extern "C" {

int fftm_get_field(fftm_problem* p, int field, void* dst, int dst_is_device, size_t bytes) {
  if (!p || !dst) return set_err(FFTM_E_INVALID, "null argument");
  size_t need;
  int rc = fftm_field_bytes(p, field, &need);
  if (rc) return rc;
  if (bytes != need) return set_err(FFTM_E_INVALID, "byte count does not match the field");
  CU(cudaSetDevice(p->ctx->device));
  if (p->esz == 8) return get_field_t<double>(p, field, dst, dst_is_device, bytes);
  return get_field_t<float>(p, field, dst, dst_is_device, bytes);
}

}  // extern "C"

template <typename T>
static int set_field_t(fftm_problem* p, int field, const void* src, int src_is_device, size_t bytes) {
  cudaStream_t s = p->ctx->stream;
  const void* from = src;
  if (!src_is_device) {
    int rc = ensure_scratch(p, bytes);
    if (rc) return rc;
    CU(cudaMemcpyAsync(p->scratch, src, bytes, cudaMemcpyHostToDevice, s));
    from = p->scratch;
  }
  T* dst[3];
  for (int q = 0; q < 3; ++q) dst[q] = field_ptr<T>(p, field == FFTM_FIELD_U ? SET_UH + p->cur : SET_WORK, q);
  if (field == FFTM_FIELD_U && p->esz == 4)
    for (int q = 0; q < 3; ++q)
      CU(cudaMemsetAsync(field_ptr<T>(p, SET_UL + p->cur, q), 0, p->comp_stride * sizeof(T), s));
  CU(launch_pack<T>((const T* const*)dst, const_cast<T*>(reinterpret_cast<const T*>(from)), p->N[0], p->N[1],
                    p->N[2], p->sy, p->sz, 1, s));
  CU(launch_mask<T>(dst, p->lo, p->hi, p->N[0], p->N[1], p->N[2], p->sy, p->sz, s));
  p->launches += 2;
  CU(cudaStreamSynchronize(s));
  return FFTM_OK;
}

extern "C" {

int fftm_set_field(fftm_problem* p, int field, const void* src, int src_is_device, size_t bytes) {
  if (!p || !src) return set_err(FFTM_E_INVALID, "null argument");
  if (field != FFTM_FIELD_U && field != FFTM_FIELD_WORK && field != FFTM_FIELD_STATE)
    return set_err(FFTM_E_INVALID, "only U, WORK and STATE are settable");
  size_t need;
  int rc = fftm_field_bytes(p, field, &need);
  if (rc) return rc;
  if (bytes != need) return set_err(FFTM_E_INVALID, "byte count does not match the field");
  CU(cudaSetDevice(p->ctx->device));
  if (field == FFTM_FIELD_STATE) {
    const void* from = src;
    if (!src_is_device) {
      rc = ensure_scratch(p, bytes);
      if (rc) return rc;
      CU(cudaMemcpyAsync(p->scratch, src, bytes, cudaMemcpyHostToDevice, p->ctx->stream));
      from = p->scratch;
    }
    if (p->esz == 8)
      CU(launch_state_io<double>(commit_params<double>(p), p->tetra, nullptr, reinterpret_cast<const double*>(from),
                                 p->ctx->stream));
    else
      CU(launch_state_io<float>(commit_params<float>(p), p->tetra, nullptr, reinterpret_cast<const float*>(from),
                                p->ctx->stream));
    p->launches++;
    CU(cudaStreamSynchronize(p->ctx->stream));
    return FFTM_OK;
  }
  if (p->esz == 8) return set_field_t<double>(p, field, src, src_is_device, bytes);
  return set_field_t<float>(p, field, src, src_is_device, bytes);
}

}  // extern "C"

template <typename T>
static int apply_t(fftm_problem* p, int op, double* norms) {
  cudaStream_t s = p->ctx->stream;
  int rc = FFTM_OK;
  switch (op) {
    case FFTM_OP_RESIDUAL: {
      // the one-pass form forced (passes 1 and a tile height): D and the norms from the
      // solver's own kernels on u^f (hi + lo), p not formed
      const bool solver_form = p->res_passes == 1 && p->res_two_pass == 0;
      rc = solver_form ? run_residual<T>(p, p->cur, false, true) : run_residual<T>(p, p->cur, true);
      if (rc) return rc;
      CU(cudaMemcpyAsync(p->hpin, p->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (norms) {
        norms[0] = p->hpin[0];
        norms[1] = p->hpin[1];
        norms[2] = error_of(p, p->hpin[0], p->hpin[1]);
      }
      return FFTM_OK;
    }
    case FFTM_OP_DT_FORWARD:
      for (int a = 0; a < 3 && !rc; ++a)
        rc = p->tf ? launch_tf(p, tf_params(p, a, 0, 0, SET_WORK, SET_WORK))
             : p->tc ? launch_tc(p, tc_params(p, a, 0, 0, SET_WORK, SET_WORK))
                     : run_pass<T>(p, a, 0, 0, SET_WORK, SET_WORK, false);
      break;
    case FFTM_OP_DT_INVERSE:
      for (int a = 2; a >= 0 && !rc; --a)
        rc = p->tf ? launch_tf(p, tf_params(p, a, 1, 0, SET_WORK, SET_WORK))
             : p->tc ? launch_tc(p, tc_params(p, a, 1, 0, SET_WORK, SET_WORK))
                     : run_pass<T>(p, a, 1, 0, SET_WORK, SET_WORK, true);
      break;
    case FFTM_OP_GREEN: {
      if (p->c0) {  // the coupled operator on the coefficients in WORK, no normalisation
        C0Params<T> G = c0_params<T>(p, true, false);
        CU(launch_green_c0<T>(G, s));
        p->launches++;
        break;
      }
      PassParams<T> P = pass_params<T>(p, 2, 0, 0, SET_WORK, SET_WORK);
      GreenParams<T> G;
      std::memset(&G, 0, sizeof(G));
      for (int q = 0; q < 3; ++q) {
        G.f[q] = field_ptr<T>(p, SET_WORK, q);
        G.gscale[q] = T(1);
        for (int a = 0; a < 3; ++a) {
          G.S2[q][a] = P.S2[q][a];
          G.C2[q][a] = P.C2[q][a];
          G.flo[q][a] = P.flo[q][a];
          G.fL[q][a] = P.fL[q][a];
        }
      }
      for (int a = 0; a < 3; ++a) {
        G.N[a] = p->N[a];
        G.hf[a] = P.hf[a];
      }
      G.sy = p->sy;
      G.sz = p->sz;
      G.two_mu0 = P.two_mu0;
      G.lam0 = P.lam0;
      G.tetra = p->tetra;
      CU(launch_green<T>(G, s));
      p->launches++;
      break;
    }
    case FFTM_OP_GREEN_UPDATE:
      // u^f = Gamma(WORK) into the current slot (low part cleared)
      if (p->esz == 4)
        for (int q = 0; q < 3; ++q)
          CU(cudaMemsetAsync(field_ptr<T>(p, SET_UL + p->cur, q), 0, p->comp_stride * sizeof(T), s));
      rc = green_apply<T>(p, SET_WORK, -1, -1, SET_UH + p->cur, -1, false);
      break;
    default:
      return set_err(FFTM_E_INVALID, "unknown op");
  }
  if (rc) return rc;
  CU(cudaStreamSynchronize(s));
  if (p->tc || p->tf) {
    int e = 0;
    CU(cudaMemcpy(&e, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      CU(cudaMemset(p->tc_err, 0, sizeof(int)));
      return set_err(FFTM_E_TIMEOUT, "a tensor-core transform pass timed out waiting for its MMAs");
    }
  }
  return FFTM_OK;
}

extern "C" {

int fftm_apply(fftm_problem* p, int op, double* norms) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  CU(cudaSetDevice(p->ctx->device));
  if (p->esz == 8) return apply_t<double>(p, op, norms);
  return apply_t<float>(p, op, norms);
}

int fftm_reset_state(fftm_problem* p) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  CU(cudaSetDevice(p->ctx->device));
  Sizes sz = sizes_of(&p->desc);
  CU(cudaMemsetAsync(p->fields, 0, sz.fields, p->ctx->stream));
  if (p->state) {
    CU(cudaMemsetAsync(p->state, 0, (size_t)(p->tetra ? 2 : 1) * p->nst * p->nvox * p->esz, p->ctx->stream));
    CU(cudaMemsetAsync(p->state_next, 0, (size_t)(p->tetra ? 2 : 1) * p->nst * p->nvox * p->esz, p->ctx->stream));
  }
  p->commit_pending = 0;
  if (p->un)
    CU(cudaMemsetAsync(p->un, 0, (size_t)(p->esz == 4 ? 6 : 3) * p->comp_stride * p->esz, p->ctx->stream));
  std::memset(&p->load_n, 0, sizeof(p->load_n));
  p->committed = 0;
  p->mixed_prev = 0;
  CU(cudaStreamSynchronize(p->ctx->stream));
  p->cur = 0;
  return FFTM_OK;
}

int fftm_set_profiling(fftm_problem* p, int enable) {
  if (!p) return set_err(FFTM_E_INVALID, "null problem");
  CU(cudaSetDevice(p->ctx->device));
  CU(cudaStreamSynchronize(p->ctx->stream));
  prof_flush(p);
  p->prof = enable != 0;
  for (int c = 0; c < FFTM_KCAT_COUNT; ++c) {
    p->prof_ms[c] = 0.0;
    p->prof_cnt[c] = 0;
  }
  return FFTM_OK;
}

int fftm_kernel_times(const fftm_problem* p, double* ms, long long* launches, int n) {
  if (!p || !ms || !launches || n < FFTM_KCAT_COUNT) return set_err(FFTM_E_INVALID, "bad arguments");
  for (int c = 0; c < FFTM_KCAT_COUNT; ++c) {
    ms[c] = p->prof_ms[c];
    launches[c] = p->prof_cnt[c];
  }
  return FFTM_OK;
}

int fftm_kernel_launches(const fftm_problem* p, long long* count) {
  if (!p || !count) return set_err(FFTM_E_INVALID, "null argument");
  *count = p->launches;
  return FFTM_OK;
}

}  // extern "C"

// ======================================================================================
// Residual evaluation that allocates nothing.
//
// Some callers may not allocate device memory at the point where they need a
// residual: code that runs while a CUDA stream is being captured into a graph
// (where a cudaMalloc would break or invalidate the capture), frameworks whose
// caching allocator or memory pool must own every device byte, and fixed-memory
// real-time loops.  fftm_residual_noalloc serves them: the caller passes u^f and
// receives D and the norms in its own device buffers, and the per-block partial
// sums of the reduction live in the file-scope array below, which the module
// loader places in every device context that loads the library (128 KiB per
// GPU, held until the process exits).
namespace {

constexpr int kNoAllocScratchDoubles = 16384;  // 128 KiB of block partials + 4 result slots
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).  Host
// code may not pass g_noalloc_scratch itself to a kernel: on the host that name
// is only a stand-in for the symbol, not a device address.
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return set_err(FFTM_E_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return set_err(FFTM_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = reinterpret_cast<double*>(ptr);
  }
  *out = g_noalloc_ptr[device];
  return FFTM_OK;
}

__global__ void k_noalloc_norms(const double* __restrict__ sums, double h1, double* __restrict__ norms) {
  const double sd = sums[0], sp = sums[1];
  norms[0] = sd;
  norms[1] = sp;
  norms[2] = sp > 0.0 ? h1 * sqrt(sd / sp) : (sd == 0.0 ? 0.0 : CUDART_INF);
}

template <typename T>
int residual_noalloc_t(fftm_problem* p, const T* u, T* D, double* norms) {
  double* scratch = nullptr;
  int rc = noalloc_scratch(p->ctx->device, &scratch);
  if (rc) return rc;
  const long long per = (long long)p->N[0] * p->N[1] * p->N[2];
  ResParams<T> R = res_params<T>(p, p->cur, nullptr, nullptr);
  for (int q = 0; q < 3; ++q) {
    R.u[q] = u + q * per;
    R.ulo[q] = nullptr;
    R.D[q] = D + q * per;
    R.p[q] = nullptr;
  }
  R.sy = p->N[0];
  R.sz = (long long)p->N[0] * p->N[1];
  const int blocks = residual_blocks<T>(R, p->tetra);
  if (2LL * blocks > kNoAllocScratchDoubles - 4)
    return set_err(FFTM_E_UNSUPPORTED, "grid too large for the no-allocation scratch (" +
                                           std::to_string(blocks) + " blocks need " + std::to_string(2 * blocks) +
                                           " doubles; the maximum is " +
                                           std::to_string(kNoAllocScratchDoubles - 4) + ")");
  R.partial = scratch;  // every block overwrites its two slots: nothing has to start at zero
  double* sums = scratch + kNoAllocScratchDoubles - 4;
  cudaStream_t s = p->ctx->stream;
  CU(launch_residual<T>(R, p->tetra, false, s, nullptr));
  CU(launch_reduce_norms(scratch, blocks, 2, sums, s));
  k_noalloc_norms<<<1, 1, 0, s>>>(sums, p->h[0], norms);
  CU(cudaGetLastError());
  p->launches += 3;
  return FFTM_OK;
}

}  // namespace

extern "C" int fftm_residual_noalloc(fftm_problem* p, const void* u_dev, void* D_dev, double* norms_dev) {
  if (!p || !u_dev || !D_dev || !norms_dev) return set_err(FFTM_E_INVALID, "null argument");
  CU(cudaSetDevice(p->ctx->device));
  if (p->esz == 8)
    return residual_noalloc_t<double>(p, reinterpret_cast<const double*>(u_dev), reinterpret_cast<double*>(D_dev),
                                      norms_dev);
  return residual_noalloc_t<float>(p, reinterpret_cast<const float*>(u_dev), reinterpret_cast<float*>(D_dev),
                                   norms_dev);
}
