// aat_api.cu -- host side of the library: number theory for Y (Sec. 4),
// digit-split planning, the recursion scheduler of Algorithm 1 with the
// memory placement of Sec. 7 (Table 3), workspace management and the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/aat.h"
#include "../../include/aat_testing.h"
#include "common.cuh"

namespace aat {

// ------------------------------------------------------------ errors

static thread_local std::string g_last_error;

static int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

static int cuda_fail(cudaError_t e, const char *where) {
  return fail(AAT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------- number theory

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t p) {
  return (uint64_t)(((unsigned __int128)a * b) % p);
}

static uint64_t powmod64(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod64(r, a, p);
    a = mulmod64(a, a, p);
    e >>= 1;
  }
  return r;
}

// Deterministic Miller-Rabin: bases 2, 3, 5, 7 are exact below 3.2e9.
static bool is_prime_u32(uint64_t n) {
  if (n < 2) return false;
  static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (uint64_t q : small) {
    if (n == q) return true;
    if (n % q == 0) return false;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint64_t a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull}) {
    uint64_t x = powmod64(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod64(x, x, n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

static uint64_t canon64(int64_t a, uint64_t p) {
  int64_t r = a % (int64_t)p;
  return (uint64_t)(r < 0 ? r + (int64_t)p : r);
}

// Euler's criterion.
static int legendre(uint64_t a, uint64_t p) {
  a %= p;
  if (a == 0) return 0;
  return powmod64(a, (p - 1) / 2, p) == 1 ? 1 : -1;
}

// Tonelli-Shanks; returns false for a non-square.
static bool sqrt_mod(uint64_t a, uint64_t p, uint64_t *root) {
  a %= p;
  if (a == 0) {
    *root = 0;
    return true;
  }
  if (legendre(a, p) != 1) return false;
  if (p % 4 == 3) {
    *root = powmod64(a, (p + 1) / 4, p);
    return true;
  }
  uint64_t q = p - 1;
  int s = 0;
  while ((q & 1) == 0) {
    q >>= 1;
    ++s;
  }
  uint64_t z = 2;
  while (legendre(z, p) != -1) ++z;
  uint64_t c = powmod64(z, q, p), t = powmod64(a, q, p), r = powmod64(a, (q + 1) / 2, p);
  int m = s;
  while (t != 1) {
    int i = 0;
    uint64_t tt = t;
    while (tt != 1) {
      tt = mulmod64(tt, tt, p);
      ++i;
      if (i >= m) return false;
    }
    uint64_t b = c;
    for (int e = 0; e < m - i - 1; ++e) b = mulmod64(b, b, p);
    m = i;
    c = mulmod64(b, b, p);
    t = mulmod64(t, c, p);
    r = mulmod64(r, b, p);
  }
  *root = r;
  return true;
}

// Algorithm 3 (SoS): a^2 + b^2 == k mod p.
static bool sos(uint64_t k, uint64_t p, uint64_t *a, uint64_t *b) {
  k %= p;
  if (legendre(k, p) >= 0) {  // k is 0 or a square
    uint64_t r;
    if (!sqrt_mod(k, p, &r)) return false;
    *a = r;
    *b = 0;
    return true;
  }
  uint64_t s = 2;
  while (legendre(s, p) == 1) ++s;  // smallest quadratic non-residue
  uint64_t c, r;
  if (!sqrt_mod(s - 1, p, &c)) return false;  // s - 1 is a square
  uint64_t rr = mulmod64(k, powmod64(s, p - 2, p), p);
  if (!sqrt_mod(rr, p, &r)) return false;
  *a = r;
  *b = mulmod64(r, c, p);
  return true;
}

ModP make_modp(uint32_t p) {
  ModP m;
  m.p = p;
  m.half = (p - 1) / 2;
  m.mu = (uint64_t)(((unsigned __int128)1 << 64) / p);
  const uint64_t two62 = (uint64_t)1 << 62;
  m.off = ((two62 + p - 1) / p) * (uint64_t)p;
  m.mu32 = (uint32_t)(((uint64_t)1 << 32) / p);
  return m;
}

static int32_t bal_host(uint64_t r, uint32_t p) {
  return r > (p - 1) / 2 ? (int32_t)((int64_t)r - (int64_t)p) : (int32_t)r;
}

// Y for the transposition over F_p (Sec. 4.2 / Prop. 4.2 with Algorithm 3).
static bool make_y_uncached(uint32_t p, YParams *y) {
  if (p % 4 == 1) {
    uint64_t i;
    if (!sqrt_mod(p - 1, p, &i)) return false;
    if (mulmod64(i, i, p) != p - 1) return false;
    y->kind = 1;
    y->a = bal_host(i, p);
    y->b = 0;
    return true;
  }
  // p = 3 mod 8: -2 is a square (Lemma 4.3), so a = 1, b = sqrt(-2) give
  // a^2 + b^2 = -1 and Y costs 2 multiplications per column pair instead of
  // 3 (the examples closing Sec. 3)
  if (p % 8 == 3) {
    uint64_t r;
    if (sqrt_mod(p - 2, p, &r) && (1 + mulmod64(r, r, p)) % p == p - 1) {
      y->kind = 2;
      y->a = 1;
      y->b = bal_host(r, p);
      return true;
    }
  }
  uint64_t a, b;
  if (!sos(p - 1, p, &a, &b)) return false;
  if ((mulmod64(a, a, p) + mulmod64(b, b, p)) % p != p - 1) return false;
  y->kind = 2;
  y->a = bal_host(a, p);
  y->b = bal_host(b, p);
  return true;
}

// Y per prime, computed once.  The remark after Algorithm 3 (Sec. 4.3)
// reuses the quadratic non-residue for several sums of squares modulo one
// prime; calls with the same p here reuse the whole Y, so the square roots
// and the two-squares search run on the first call with p only.
static std::mutex g_y_mu;
static std::map<uint32_t, YParams> g_y_cache;

static bool make_y(uint32_t p, YParams *y) {
  {
    std::lock_guard<std::mutex> lock(g_y_mu);
    auto it = g_y_cache.find(p);
    if (it != g_y_cache.end()) {
      *y = it->second;
      return true;
    }
  }
  if (!make_y_uncached(p, y)) return false;
  std::lock_guard<std::mutex> lock(g_y_mu);
  if (g_y_cache.size() < 4096) g_y_cache[p] = *y;
  return true;
}

// Signed base-2^b digits of balanced residues: the fewest digits whose top
// digit stays exact in BF16 (|d| <= 256), then the smallest digit products.
static DigitSpec make_digits(uint32_t p) {
  DigitSpec best;
  std::memset(&best, 0, sizeof(best));
  int64_t best_prod = -1;
  for (int b : {8, 9, 7}) {
    DigitSpec d;
    std::memset(&d, 0, sizeof(d));
    d.b = b;
    int64_t X = (p - 1) / 2;
    int L = 1;
    while (X > 256 && L < 8) {
      d.dmax[L - 1] = 1 << (b - 1);
      X = (X + (1 << (b - 1))) >> b;
      ++L;
    }
    d.dmax[L - 1] = (int)std::max<int64_t>(X, 1);
    d.L = L;
    int64_t mx = 0;
    for (int i = 0; i < L; ++i) mx = std::max<int64_t>(mx, d.dmax[i]);
    const int64_t prod = mx * mx;
    if (best_prod < 0 || d.L < best.L || (d.L == best.L && prod < best_prod)) {
      best = d;
      best_prod = prod;
    }
  }
  // Pair sums: x_i y_j + x_j y_i = (x_i + x_j)(y_i + y_j) - x_i y_i - x_j y_j, so
  // L + L(L-1)/2 plane products replace L^2 when every sum stays exact in
  // bf16 (|d_i + d_j| <= 256).
  bool ok = best.L >= 2 && best.L <= 4;
  for (int i = 0; ok && i < best.L; ++i)
    for (int j = i + 1; j < best.L; ++j)
      if (best.dmax[i] + best.dmax[j] > 256) ok = false;
  best.nsum = 0;
  if (ok)
    for (int i = 0; i < best.L; ++i)
      for (int j = i + 1; j < best.L; ++j) {
        best.si[best.nsum] = i;
        best.sj[best.nsum] = j;
        ++best.nsum;
      }
  return best;
}

// ------------------------------------------------------- device state

struct DeviceState {
  void *ws = nullptr;
  size_t ws_size = 0;
  int32_t *status = nullptr;
  // buffers of the end-to-end host entry point
  void *e2e_a = nullptr, *e2e_c = nullptr;
  size_t e2e_a_size = 0, e2e_c_size = 0;
  cudaStream_t e2e_stream = nullptr;
  cudaStream_t e2e_stream2 = nullptr;  // copies rows that are final early
  cudaEvent_t e2e_split = nullptr;
  cudaEvent_t e2e_a11 = nullptr, e2e_rest = nullptr;  // copies of A in
  std::vector<cudaEvent_t> e2e_bands;  // row bands of the rest of A in
};

static std::mutex g_state_mu;
static std::map<int, DeviceState> g_states;

static DeviceState &state() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_states[dev];
}

int32_t *device_status_ptr() {
  std::lock_guard<std::mutex> lock(g_state_mu);
  DeviceState &s = state();
  if (!s.status) {
    if (cudaMalloc(&s.status, sizeof(int32_t)) != cudaSuccess) return nullptr;
    cudaMemset(s.status, 0, sizeof(int32_t));
  }
  return s.status;
}

// Test hook: workspace requests above this many bytes fail with AAT_ENOMEM
// as a failed cudaMalloc would, before any CUDA call (SIZE_MAX: no limit).
static std::atomic<size_t> g_alloc_limit{SIZE_MAX};
// aat_set_workspace_limit: products whose fast schedule needs more workspace
// run the low-memory plane passes (SIZE_MAX: no limit).
static std::atomic<size_t> g_ws_limit{SIZE_MAX};

static int ensure_workspace(size_t bytes, void **out) {
  if (bytes > g_alloc_limit.load())
    return fail(AAT_ENOMEM, "workspace allocation of " + std::to_string(bytes) +
                                " bytes refused (test allocation limit " +
                                std::to_string(g_alloc_limit.load()) + ")");
  std::lock_guard<std::mutex> lock(g_state_mu);
  DeviceState &s = state();
  if (s.ws_size < bytes) {
    if (s.ws) {
      cudaDeviceSynchronize();
      cudaFree(s.ws);
      s.ws = nullptr;
      s.ws_size = 0;
    }
    size_t want = bytes + (bytes >> 4);
    cudaError_t e = cudaMalloc(&s.ws, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(AAT_ENOMEM, "workspace allocation of " + std::to_string(want) + " bytes failed");
    }
    s.ws_size = want;
  }
  *out = s.ws;
  return AAT_OK;
}

// ---------------------------------------------------- instrumentation

struct ProfRec {
  int cls;
  cudaStream_t st;
  cudaEvent_t a, b;
  double work;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(int cls, cudaStream_t st, double work) : idx(-1) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // no timing events inside a graph capture
  }
  ProfRec r{cls, st, pool_event(), pool_event(), work};
  cudaEventRecord(r.a, st);
  g_prof.push_back(r);
  idx = (int)g_prof.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx < 0) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (idx < (int)g_prof.size()) cudaEventRecord(g_prof[idx].b, g_prof[idx].st);
}

// ---------------------------------------------------------- the plan

// Bump allocator over the workspace with a dry-run mode that only measures.
struct Arena {
  char *base = nullptr;
  size_t used = 0, peak = 0;
  bool dry = true;
  void *get(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    peak = std::max(peak, used);
    return dry ? nullptr : (void *)(base + off);
  }
};

struct Ctx {
  ModP m;
  YParams y;
  DigitSpec ds;
  uint32_t leaf;     // AAT_LEAF_TC / AAT_LEAF_SIMT
  int exact_bits;
  cudaStream_t st;
  Arena ar;
  aatx_plan_stats_t *stats;  // optional counters
  int err = AAT_OK;
  // optional: recorded on `st` as soon as rows [split_row, n) of C are final
  // (after the top level's post-additions; at the end when C is padded)
  cudaEvent_t split_ev = nullptr;
  int top_levels = -1;
  int64_t split_row = 0;
  int form = 0;  // leaf kernel form (TcLeafArgs::form)
  // optional (end-to-end path): A11's and the rest of A's copies to the
  // device complete at these events; the stream waits for them.  The rest
  // may also come in nbands row bands (rows [b h / nbands, (b+1) h / nbands)
  // of A12 and of the bottom half, event in_bands[b]): the top level's
  // S-block kernel then runs band by band as they arrive.
  cudaEvent_t in_a11 = nullptr, in_rest = nullptr;
  const cudaEvent_t *in_bands = nullptr;
  int nbands = 0;
  uint32_t alpha = 1;  // scale of every product (the SYRK update's alpha)
  bool wino = false;   // last level's P3, P4 by Winograd's form (AAT_WINOGRAD)
  // low-memory plane passes (AAT_LOW_MEMORY): every leaf product runs as
  // passes over windows of pass_w planes of its operands' plane sequence
  bool passes = false;
  int pass_w = 1;
};

static Planes planes_for(const DigitSpec &ds, int64_t rows, int64_t cols) {
  Planes P;
  std::memset(&P, 0, sizeof(P));
  P.rows = rows;
  P.cols = cols;
  P.kstride = (cols + 7) / 8 * 8;
  P.nbase = ds.L;
  P.nsum = ds.nsum;
  P.L = ds.L + ds.nsum;
  for (int q = 0; q < ds.nsum; ++q) {
    P.si[q] = (int8_t)ds.si[q];
    P.sj[q] = (int8_t)ds.sj[q];
  }
  return P;
}

static Planes planes_alloc(Ctx &c, int64_t rows, int64_t cols) {
  Planes P = planes_for(c.ds, rows, cols);
  P.ptr = (__nv_bfloat16 *)c.ar.get((size_t)P.L * rows * P.kstride * 2);
  return P;
}

static Planes no_planes() {
  Planes P;
  std::memset(&P, 0, sizeof(P));
  return P;
}

// The low-memory plane passes apply to the tensor-core leaf with the
// pair-sum digit form, where every plane product reads one plane of each
// operand (plane q of X with plane q of Y): a pass over the plane window
// [q0, q0 + w) needs only those w planes of each operand.
static bool pass_mode(const Ctx &c) {
  return c.passes && c.leaf == AAT_LEAF_TC && c.ds.nsum > 0;
}

static int plane_count(const Ctx &c) { return c.ds.L + c.ds.nsum; }

// Planes q0 .. q0 + w - 1 of an r x c block, in the arena.
static Planes planes_window(Ctx &c, int64_t rows, int64_t cols, int q0, int w) {
  Planes P = planes_for(c.ds, rows, cols);
  P.q0 = q0;
  P.L = w;
  P.ptr = (__nv_bfloat16 *)c.ar.get((size_t)w * rows * P.kstride * 2);
  return P;
}

// An operand of a leaf product: an int32 residue block and/or its planes.
struct Operand {
  const int32_t *x;
  int64_t ld;
  Planes pl;  // pl.L == 0: not split yet
};

static bool check(Ctx &c, cudaError_t e, const char *where) {
  if (e != cudaSuccess && c.err == AAT_OK) c.err = cuda_fail(e, where);
  return c.err == AAT_OK;
}

// out <- alpha X Y^T + beta out (M x N, inner K) mod p, alpha = c.alpha;
// lower: only i >= j.  beta 0 stores the product, 1 accumulates.
static void count_leaf(Ctx &c, int64_t M, int64_t N, int64_t K, int lower) {
  if (c.stats) {
    if (lower) {
      c.stats->syrk_leaves++;
      c.stats->ring_macs += (double)M * (double)(M + 1) / 2.0 * (double)K;
    } else {
      c.stats->general_products++;
      c.stats->ring_macs += (double)M * (double)N * (double)K;
    }
  }
}

// The tensor-core leaf's arguments for out <- alpha X Y^T + beta out from
// the digit planes of X (M x K) and Y (N x K).
static TcLeafArgs tc_args(const Ctx &c, const Planes &x, const Planes &y, int64_t M, int64_t N,
                          int64_t K, int32_t *out, int64_t ldo, int lower, uint32_t beta) {
  TcLeafArgs a;
  a.x = x;
  a.y = y;
  a.dx = c.ds;
  a.dy = c.ds;
  a.M = M;
  a.N = N;
  a.K = K;
  a.out = out;
  a.ldo = ldo;
  a.lower = lower;
  a.lin = lin_of(c.alpha, beta, c.m.p);
  a.exact_bits = c.exact_bits;
  a.form = c.form;
  return a;
}

static void leaf(Ctx &c, Operand X, Operand Y, bool same, int64_t M, int64_t N, int64_t K,
                 int32_t *out, int64_t ldo, int lower, uint32_t beta) {
  const Lin lin = lin_of(c.alpha, beta, c.m.p);
  count_leaf(c, M, N, K, lower);
  if (c.leaf == AAT_LEAF_SIMT) {
    if (!c.ar.dry)
      check(c, launch_leaf_simt(X.x, X.ld, Y.x, Y.ld, M, N, K, out, ldo, lower, lin, c.m,
                                c.st),
            "leaf (CUDA cores)");
    return;
  }
  if (c.leaf == AAT_LEAF_I8) {
    const size_t mark = c.ar.used;
    void *ws = c.ar.get(leaf_i8_workspace(M, N, K, c.m.p));
    if (!c.ar.dry)
      check(c, launch_leaf_i8(X.x, X.ld, Y.x, Y.ld, M, N, K, out, ldo, lower, lin, c.m, ws,
                              c.st),
            "leaf (INT8 mma.sync)");
    c.ar.used = mark;
    return;
  }
  if (c.leaf == AAT_LEAF_F64) {
    if (!c.ar.dry)
      check(c, launch_leaf_f64(X.x, X.ld, Y.x, Y.ld, M, N, K, out, ldo, lower, lin, c.m,
                               c.st),
            "leaf (FP64 mma.sync)");
    return;
  }
  const size_t mark = c.ar.used;
  if (pass_mode(c) && X.pl.L == 0 && (same || Y.pl.L == 0)) {
    // low-memory plane passes: split a window of planes, run its plane
    // products, accumulate (the first pass with live terms takes beta)
    // a product of an operand by itself splits one operand per pass, so its
    // windows are twice as wide in the same workspace
    const int Q = plane_count(c), W = same ? 2 * c.pass_w : c.pass_w;
    bool first = true;
    for (int q0 = 0; q0 < Q; q0 += W) {
      const int w = std::min(W, Q - q0);
      const size_t mk = c.ar.used;
      Planes px = planes_window(c, M, K, q0, w), py = px;
      if (!same) py = planes_window(c, N, K, q0, w);
      const TcLeafArgs a = tc_args(c, px, py, M, N, K, out, ldo, lower, first ? beta : 1);
      if (!c.ar.dry && c.err == AAT_OK && leaf_tc_terms(a, c.m) > 0) {
        check(c, launch_split(X.x, X.ld, M, K, c.m, c.ds.b, px, c.st), "split");
        if (!same) check(c, launch_split(Y.x, Y.ld, N, K, c.m, c.ds.b, py, c.st), "split");
        check(c, launch_leaf_tc(a, c.m, c.st), "leaf (tensor cores, plane pass)");
        first = false;
      }
      c.ar.used = mk;
    }
    if (!c.ar.dry && first && beta == 0)  // every term vanished mod p
      check(c, cudaMemset2DAsync(out, (size_t)ldo * 4, 0, (size_t)N * 4, (size_t)M, c.st),
            "zero product");
    c.ar.used = mark;
    return;
  }
  if (X.pl.L == 0) {
    X.pl = planes_alloc(c, M, K);
    if (!c.ar.dry) check(c, launch_split(X.x, X.ld, M, K, c.m, c.ds.b, X.pl, c.st), "split");
  }
  if (same) {
    Y.pl = X.pl;
  } else if (Y.pl.L == 0) {
    Y.pl = planes_alloc(c, N, K);
    if (!c.ar.dry) check(c, launch_split(Y.x, Y.ld, N, K, c.m, c.ds.b, Y.pl, c.st), "split");
  }
  if (!c.ar.dry && c.err == AAT_OK)
    check(c, launch_leaf_tc(tc_args(c, X.pl, Y.pl, M, N, K, out, ldo, lower, beta), c.m, c.st),
          "leaf (tensor cores)");
  c.ar.used = mark;
}

// The operands of one level's products after the S-block step (K1).
struct LevelOps {
  Operand oS1, oS2, oS4, oA22;
  Planes pA11, pA12, pS3;  // planes of A11, A12, S3 (last level, tensor-core leaf)
};

// Step 1 of a level: S1..S4 (4 additions, 2 products by Y) in one pass over
// A.  S3 is written as int32 to S3 (row stride ldS3) unless it is needed
// only as digit planes (last level, tensor-core leaf; S3 may be null then).
// pA11: digit planes of A11 already split (the end-to-end path computes P1
// before the rest of A arrives), or none.
static LevelOps sblocks_step(Ctx &c, const int32_t *A, int64_t lda, int64_t h, int64_t kap,
                             int32_t *S3, int64_t ldS3, bool last, Planes pA11 = Planes{},
                             bool wino = false, bool banded = false) {
  const bool tc = (c.leaf == AAT_LEAF_TC);
  const int32_t *A22 = A + h * lda + kap;
  SKernelOut o;
  std::memset(&o, 0, sizeof(o));
  o.s[2] = (tc && last) ? nullptr : S3;
  o.lds[2] = ldS3;
  LevelOps L;
  L.oS1 = Operand{nullptr, 0, no_planes()};
  L.oS2 = L.oS1;
  L.oS4 = L.oS1;
  L.oA22 = Operand{A22, lda, no_planes()};
  L.pA11 = L.pA12 = L.pS3 = no_planes();
  if (tc) {
    if (wino) {
      // Winograd's form forms its own operand blocks from int32 S1, S2, S4
      // (and from A22 itself)
      for (int q : {0, 1, 3}) {
        o.s[q] = (int32_t *)c.ar.get((size_t)h * kap * 4);
        o.lds[q] = kap;
      }
      L.oS1 = Operand{o.s[0], kap, no_planes()};
      L.oS2 = Operand{o.s[1], kap, no_planes()};
      L.oS4 = Operand{o.s[3], kap, no_planes()};
    } else {
      o.sp[0] = L.oS1.pl = planes_alloc(c, h, kap);
      o.sp[1] = L.oS2.pl = planes_alloc(c, h, kap);
      o.sp[3] = L.oS4.pl = planes_alloc(c, h, kap);
      o.a22 = L.oA22.pl = planes_alloc(c, h, kap);
    }
    if (last) {
      if (pA11.L)
        L.pA11 = pA11;
      else
        o.a11 = L.pA11 = planes_alloc(c, h, kap);
      o.a12 = L.pA12 = planes_alloc(c, h, kap);
      o.sp[2] = L.pS3 = planes_alloc(c, h, kap);
    }
  } else {
    for (int q : {0, 1, 3}) {
      o.s[q] = (int32_t *)c.ar.get((size_t)h * kap * 4);
      o.lds[q] = kap;
    }
    L.oS1.x = o.s[0];
    L.oS1.ld = kap;
    L.oS2.x = o.s[1];
    L.oS2.ld = kap;
    L.oS4.x = o.s[3];
    L.oS4.ld = kap;
  }
  if (!c.ar.dry && banded) {
    // each band as soon as its rows of A are on the device
    for (int b = 0; b < c.nbands && c.err == AAT_OK; ++b) {
      const int64_t r0 = h * b / c.nbands, r1 = h * (b + 1) / c.nbands;
      check(c, cudaStreamWaitEvent(c.st, c.in_bands[b], 0), "wait for A");
      check(c, launch_sblocks(A, lda, h, kap, c.m, c.y, c.ds.b, o, c.st, r0, r1), "sblocks");
    }
  } else if (!c.ar.dry) {
    check(c, launch_sblocks(A, lda, h, kap, c.m, c.y, c.ds.b, o, c.st), "sblocks");
  }
  return L;
}

static void count_level(Ctx &c) {
  if (c.stats) {
    c.stats->recursive_products += 3;
    c.stats->block_additions += 9;
    c.stats->half_additions += 3;
  }
}

// Steps 2-5 of a last level with Winograd's form for the general products:
// P4^T = S2 S1^T and P3 = A22 S4^T each become seven products of half the
// size (operand blocks from one pass over S2, S1, A22, S4), which run in one
// persistent launch together with the symmetric products `sym` (P5, and P1
// unless it ran first); the seven additions after them write C22 and C21.
static void wino_products(Ctx &c, const LevelOps &L, const int32_t *A22, int64_t lda, int64_t h,
                          int64_t kap, int32_t *C21, int32_t *C22, int64_t ldc,
                          const TcLeafArgs *sym, int nsym) {
  const int64_t R = h / 2, Kq = kap / 2, ldw = (R + 3) / 4 * 4;
  WinoPlanes w[4];  // left and right operands of P4^T, then of P3
  for (WinoPlanes &wp : w)
    for (Planes &q : wp.q) q = planes_alloc(c, R, Kq);
  int32_t *W4 = (int32_t *)c.ar.get((size_t)7 * R * ldw * 4);
  int32_t *W3 = (int32_t *)c.ar.get((size_t)7 * R * ldw * 4);
  if (!c.ar.dry && c.err == AAT_OK) {
    check(c, launch_wino_operands(L.oS2.x, L.oS2.ld, R, Kq, c.m, c.ds.b, false, w[0], c.st),
          "Winograd operands");
    check(c, launch_wino_operands(L.oS1.x, L.oS1.ld, R, Kq, c.m, c.ds.b, true, w[1], c.st),
          "Winograd operands");
    check(c, launch_wino_operands(A22, lda, R, Kq, c.m, c.ds.b, false, w[2], c.st),
          "Winograd operands");
    check(c, launch_wino_operands(L.oS4.x, L.oS4.ld, R, Kq, c.m, c.ds.b, true, w[3], c.st),
          "Winograd operands");
  }
  // products W_q = left[lx[q]] right[ry[q]]^T: X11 Y11^T, X12 Y12^T,
  // S4 Y22^T, X22 V4^T, S1 V1^T, S2 V2^T, S3 V3^T
  static const int lx[7] = {0, 1, 6, 2, 3, 4, 5}, ry[7] = {0, 1, 2, 6, 3, 4, 5};
  TcLeafArgs fa[16];
  int n = 0;
  for (int side = 0; side < 2; ++side) {
    int32_t *W = side ? W3 : W4;
    for (int q = 0; q < 7; ++q) {
      fa[n] = tc_args(c, w[2 * side].q[lx[q]], w[2 * side + 1].q[ry[q]], R, R, Kq,
                      W + (size_t)q * R * ldw, ldw, 0, 0);
      count_leaf(c, R, R, Kq, 0);
      ++n;
    }
  }
  for (int q = 0; q < nsym; ++q) {
    fa[n++] = sym[q];
    count_leaf(c, sym[q].M, sym[q].N, sym[q].K, sym[q].lower);
  }
  if (c.ar.dry || c.err != AAT_OK) return;
  check(c, launch_leaf_tc_multi(fa, n, c.m, c.st), "leaf (tensor cores, Winograd products)");
  check(c, launch_wino_combine(W4, ldw, R * ldw, C22, ldc, R, R, c.m, c.st), "Winograd sums");
  check(c, launch_wino_combine(W3, ldw, R * ldw, C21, ldc, R, R, c.m, c.st), "Winograd sums");
}

// The independent leaf products of a last level in one launch or one launch
// per product: AAT_LEAF_FUSE=1 / 0 forces either, otherwise the launcher
// decides from the idle share of the separate launches' last waves.
static int fuse_override() {
  static const int v = [] {
    const char *e = getenv("AAT_LEAF_FUSE");
    return e ? (atoi(e) != 0 ? 1 : 0) : -1;
  }();
  return v;
}

// Low(A A^T) mod p -> Low(C) by Algorithm 1 with `levels` levels (times
// c.alpha).  n must be divisible by 2^levels and k by 2^levels (2^(levels+1)
// for a kind-2 Y).  `ap` optionally holds the digit planes of A
// (tensor-core leaf).  Memory placement of Table 3 (Sec. 7).
static void rec_passes(Ctx &c, const int32_t *A, int64_t lda, int64_t n, int64_t k, int32_t *C,
                       int64_t ldc, int levels);

static void rec(Ctx &c, const int32_t *A, int64_t lda, int64_t n, int64_t k, int32_t *C,
                int64_t ldc, int levels, Planes ap) {
  if (c.err != AAT_OK) return;
  if (levels == 0 || n < 2 || k < 2) {
    Operand X{A, lda, ap};
    leaf(c, X, X, true, n, n, k, C, ldc, 1, 0);
    return;
  }
  if (pass_mode(c)) {
    rec_passes(c, A, lda, n, k, C, ldc, levels);
    return;
  }
  const int64_t h = n / 2, kap = k / 2;
  int32_t *C11 = C, *C12 = C + h, *C21 = C + h * ldc, *C22 = C + h * ldc + h;
  const int32_t *A11 = A, *A12 = A + kap;
  const bool last = (levels == 1);
  const size_t mark = c.ar.used;
  count_level(c);
  // End-to-end path: A11 arrives first, so P1 = Low(A11 A11^T) runs while
  // the rest of A is copied in (step 5 moved ahead; C11 is not touched by
  // steps 1-4, and the post-additions read P1 from it as before).
  const bool p1_first = c.in_rest && levels == c.top_levels;
  Planes pA11_early = no_planes();
  if (p1_first) {
    if (!c.ar.dry) cudaStreamWaitEvent(c.st, c.in_a11, 0);
    if (c.leaf == AAT_LEAF_TC && last) {
      pA11_early = planes_alloc(c, h, kap);
      if (!c.ar.dry)
        check(c, launch_split(A11, lda, h, kap, c.m, c.ds.b, pA11_early, c.st), "split");
    }
    rec(c, A11, lda, h, kap, C11, ldc, levels - 1, pA11_early);
    if (!c.ar.dry && c.nbands == 0) cudaStreamWaitEvent(c.st, c.in_rest, 0);
  }
  const bool banded = p1_first && c.nbands > 0;
  // S3: the input of the recursive product P5.  Table 3 keeps it in C21
  // (needs kappa <= h, i.e. k <= n); otherwise it takes workspace.
  int32_t *S3;
  int64_t ldS3;
  if (kap <= h) {
    S3 = C21;
    ldS3 = ldc;
  } else {
    S3 = (int32_t *)c.ar.get((size_t)h * kap * 4);
    ldS3 = kap;
  }
  // Winograd's form for the last level's general products (blocks of even
  // sides only)
  const bool wino = last && c.leaf == AAT_LEAF_TC && c.wino && h % 2 == 0 && kap % 2 == 0;
  // 1. S1..S4 (4 additions, 2 products by Y) in one pass over A
  const LevelOps L = sblocks_step(c, A, lda, h, kap, S3, ldS3, last, pA11_early, wino, banded);
  // everything after the S blocks may read any row of A
  if (banded && !c.ar.dry) cudaStreamWaitEvent(c.st, c.in_rest, 0);
  // 2-5 at the last level: P4^T, P5, P3 and P1 read only digit planes
  // written by step 1 and write four different blocks of C, so they may run
  // as one persistent launch over the tiles of all four
  TcLeafArgs fa[4];
  int nfa = 0;
  if (last && c.leaf == AAT_LEAF_TC) {
    fa[nfa++] = tc_args(c, L.oS2.pl, L.oS1.pl, h, h, kap, C22, ldc, 0, 0);
    fa[nfa++] = tc_args(c, L.pS3, L.pS3, h, h, kap, C12, ldc, 1, 0);
    fa[nfa++] = tc_args(c, L.oA22.pl, L.oS4.pl, h, h, kap, C21, ldc, 0, 0);
    if (!p1_first) fa[nfa++] = tc_args(c, L.pA11, L.pA11, h, h, kap, C11, ldc, 1, 0);
  }
  const int fo = fuse_override();
  if (wino) {
    const TcLeafArgs sym[2] = {fa[1], fa[nfa - 1]};  // P5, and P1 unless it ran first
    wino_products(c, L, A + h * lda + kap, lda, h, kap, C21, C22, ldc, sym, p1_first ? 1 : 2);
  } else if (nfa > 0 && (fo == 1 || (fo < 0 && leaf_tc_fuse_pays(fa, nfa)))) {
    for (int q = 0; q < nfa; ++q) count_leaf(c, fa[q].M, fa[q].N, fa[q].K, fa[q].lower);
    if (!c.ar.dry && c.err == AAT_OK)
      check(c, launch_leaf_tc_multi(fa, nfa, c.m, c.st), "leaf (tensor cores, P1 P3 P4 P5)");
  } else {
    // 2. P4^T = S2 S1^T -> C22
    leaf(c, L.oS2, L.oS1, false, h, h, kap, C22, ldc, 0, 0);
    // 3. P5 = Low(S3 S3^T) -> C12
    rec(c, S3, ldS3, h, kap, C12, ldc, levels - 1, L.pS3);
    // 4. P3 = A22 S4^T -> C21 (S3 is no longer needed)
    leaf(c, L.oA22, L.oS4, false, h, h, kap, C21, ldc, 0, 0);
    // 5. P1 = Low(A11 A11^T) -> C11
    if (!p1_first) rec(c, A11, lda, h, kap, C11, ldc, levels - 1, L.pA11);
  }
  // 6. U1 = P1 + P5, U2 = U1 + P4, U4 = U2 + P3 -> C21, U5 = Low(U2 + P4^T) -> C22
  if (!c.ar.dry) check(c, launch_postadd(C11, ldc, C12, C21, C22, ldc, h, c.m, c.st), "postadd");
  // rows [h, n) of the top level (C21 = U4, Low(C22) = Low(U5)) are final
  if (c.split_ev && levels == c.top_levels && !c.ar.dry && c.err == AAT_OK)
    cudaEventRecord(c.split_ev, c.st);
  // 7-8. P2 = Low(A12 A12^T), U3 = P1 + P2 -> C11
  if (last) {
    Operand X{A12, lda, L.pA12};
    leaf(c, X, X, true, h, h, kap, C11, ldc, 1, 1);  // accumulates onto P1
  } else {
    rec(c, A12, lda, h, kap, C12, ldc, levels - 1, no_planes());
    if (!c.ar.dry) check(c, launch_add_low(C11, ldc, C12, ldc, h, c.m, c.st), "add_low");
  }
  c.ar.used = mark;
}

// One level of Algorithm 1 in the low-memory schedule: Table 3's placement
// and order (Sec. 7), with every leaf product in plane passes.  The S blocks
// are int32 residues in the blocks of C that Table 3 assigns them (S1 -> C21,
// S2 -> C12; then S3 -> C21 over S1 and S4 -> C11), each product reads them
// there and writes where Table 3 puts it (P4^T -> C22, P5 -> C12 over S2,
// P3 -> C21 over S3, P1 -> C11 over S4), so the only workspace is one pass's
// digit planes (leaf()).  The S-block kernel forms the S blocks from A in
// two passes over A (S1 and S2; then S3 and S4).  With k > n the S blocks do
// not fit into C's blocks (Table 3 needs k <= n): two h x kappa int32
// buffers of workspace hold them instead (S1, S2, then S3, S4).
static void rec_passes(Ctx &c, const int32_t *A, int64_t lda, int64_t n, int64_t k, int32_t *C,
                       int64_t ldc, int levels) {
  const int64_t h = n / 2, kap = k / 2;
  int32_t *C11 = C, *C12 = C + h, *C21 = C + h * ldc, *C22 = C + h * ldc + h;
  const int32_t *A11 = A, *A12 = A + kap, *A22 = A + h * lda + kap;
  const bool last = (levels == 1);
  const size_t mark = c.ar.used;
  count_level(c);
  // where S1 / S3 and S2 / S4 live
  int32_t *Sa = C21, *Sb = C12;
  int64_t lda_s = ldc, ldb_s = ldc;
  if (kap > h) {
    Sa = (int32_t *)c.ar.get((size_t)h * kap * 4);
    Sb = (int32_t *)c.ar.get((size_t)h * kap * 4);
    lda_s = ldb_s = kap;
  }
  auto sblocks = [&](int q0, int32_t *p0, int64_t l0, int q1, int32_t *p1, int64_t l1) {
    if (c.ar.dry || c.err != AAT_OK) return;
    SKernelOut o;
    std::memset(&o, 0, sizeof(o));
    o.s[q0] = p0;
    o.lds[q0] = l0;
    o.s[q1] = p1;
    o.lds[q1] = l1;
    check(c, launch_sblocks(A, lda, h, kap, c.m, c.y, c.ds.b, o, c.st), "sblocks");
  };
  // 1-2. S1 = (A21 - A11) Y -> C21, S2 = A22 - A21 Y -> C12
  sblocks(0, Sa, lda_s, 1, Sb, ldb_s);
  // 3. P4^T = S2 S1^T -> C22
  leaf(c, Operand{Sb, ldb_s, no_planes()}, Operand{Sa, lda_s, no_planes()}, false, h, h, kap,
       C22, ldc, 0, 0);
  // 4, 6. S3 = S1 - A22 -> C21 (over S1), S4 = S3 + A12 -> C11 (or workspace)
  int32_t *S4 = (kap > h) ? Sb : C11;
  const int64_t ld4 = (kap > h) ? ldb_s : ldc;
  sblocks(2, Sa, lda_s, 3, S4, ld4);
  // 5. P5 = Low(S3 S3^T) -> C12 (over S2)
  rec(c, Sa, lda_s, h, kap, C12, ldc, levels - 1, no_planes());
  // 7. P3 = A22 S4^T -> C21 (over S3)
  leaf(c, Operand{A22, lda, no_planes()}, Operand{S4, ld4, no_planes()}, false, h, h, kap, C21,
       ldc, 0, 0);
  // 8. P1 = Low(A11 A11^T) -> C11 (over S4)
  rec(c, A11, lda, h, kap, C11, ldc, levels - 1, no_planes());
  // 9-12. U1 = P1 + P5, U2 = U1 + P4, U4 = U2 + P3 -> C21, Low(U5) -> C22
  if (!c.ar.dry) check(c, launch_postadd(C11, ldc, C12, C21, C22, ldc, h, c.m, c.st), "postadd");
  if (c.split_ev && levels == c.top_levels && !c.ar.dry && c.err == AAT_OK)
    cudaEventRecord(c.split_ev, c.st);
  // 13-14. P2 = Low(A12 A12^T), U3 = P1 + P2 -> C11
  if (last) {
    Operand X{A12, lda, no_planes()};
    leaf(c, X, X, true, h, h, kap, C11, ldc, 1, 1);  // accumulates onto P1
  } else {
    rec(c, A12, lda, h, kap, C12, ldc, levels - 1, no_planes());
    if (!c.ar.dry) check(c, launch_add_low(C11, ldc, C12, ldc, h, c.m, c.st), "add_low");
  }
  c.ar.used = mark;
}

// Low(C) <- alpha Low(A A^T) + beta Low(C) mod p, alpha = c.alpha (the SYRK
// form, Sec. 7, Table 4).  The schedule of Table 4: C12 and one h x h
// temporary (tmp) hold intermediate blocks, the strictly lower part of C22
// is saved transposed in the upper triangle of C11 (its diagonal in an
// h-vector: Up(C11) includes the diagonal, which C11 itself still needs), P3
// and P2 take beta C21 and beta C11 in their epilogues, U5 takes beta C22.
// P5 and P1 are plain products (beta = 0) by `rec`; P2 is this update,
// recursively, on (A12, C11).
static void syrk_rec(Ctx &c, const int32_t *A, int64_t lda, int64_t n, int64_t k, int32_t *C,
                     int64_t ldc, int levels, const MulConst &beta) {
  if (c.err != AAT_OK) return;
  if (levels == 0 || n < 2 || k < 2) {
    Operand X{A, lda, no_planes()};
    leaf(c, X, X, true, n, n, k, C, ldc, 1, beta.w);
    return;
  }
  const int64_t h = n / 2, kap = k / 2;
  int32_t *C11 = C, *C12 = C + h, *C21 = C + h * ldc, *C22 = C + h * ldc + h;
  const int32_t *A11 = A, *A12 = A + kap;
  const bool last = (levels == 1);
  const size_t mark = c.ar.used;
  count_level(c);
  int32_t *tmp = (int32_t *)c.ar.get((size_t)h * h * 4);
  int32_t *dg = (int32_t *)c.ar.get((size_t)h * 4);
  // S3 (when needed as int32) lives in tmp until P1 takes it (k <= n)
  int32_t *S3;
  int64_t ldS3;
  if (kap <= h) {
    S3 = tmp;
    ldS3 = h;
  } else {
    S3 = (int32_t *)c.ar.get((size_t)h * kap * 4);
    ldS3 = kap;
  }
  const LevelOps L = sblocks_step(c, A, lda, h, kap, S3, ldS3, last);
  // Up(C11) <- Low(C22)^T (strictly), diag(C22) -> dg
  if (!c.ar.dry) check(c, launch_save_c22(C11, C22, ldc, h, dg, c.st), "save C22");
  // P4^T = alpha S2 S1^T -> C22
  leaf(c, L.oS2, L.oS1, false, h, h, kap, C22, ldc, 0, 0);
  // P5 = alpha Low(S3 S3^T) -> C12
  rec(c, S3, ldS3, h, kap, C12, ldc, levels - 1, L.pS3);
  // P3 = alpha A22 S4^T + beta C21 -> C21
  leaf(c, L.oA22, L.oS4, false, h, h, kap, C21, ldc, 0, beta.w);
  // P1 = alpha Low(A11 A11^T) -> tmp (S3 is no longer needed)
  rec(c, A11, lda, h, kap, tmp, h, levels - 1, L.pA11);
  // U1 = P1 + P5, U2 = U1 + P4, U4 = U2 + P3 -> C21,
  // U5 = Low(U2 + P4^T) + beta Low(C22 before) -> C22
  const SyrkSave sv{C11, dg, beta};
  if (!c.ar.dry) check(c, launch_postadd(tmp, h, C12, C21, C22, ldc, h, c.m, c.st, &sv), "postadd");
  // P2 = alpha A12 A12^T + beta C11 -> C11, then U3 = P1 + P2 -> C11
  if (last) {
    Operand X{A12, lda, L.pA12};
    leaf(c, X, X, true, h, h, kap, C11, ldc, 1, beta.w);
  } else {
    syrk_rec(c, A12, lda, h, kap, C11, ldc, levels - 1, beta);
  }
  if (!c.ar.dry) check(c, launch_add_low(C11, ldc, tmp, h, h, c.m, c.st), "add_low");
  c.ar.used = mark;
}

// ------------------------------------------------------------ tuning table

// Tuned choices for Low(A A^T) mod p on the tensor-core leaf, per (n, k, p):
// recursion levels, leaf kernel form (TcLeafArgs::form) and digit-product
// form.  Filled by aat_tune_modp or aat_tune_load; consulted whenever the
// flags leave these choices open.
struct TuneVal {
  int levels, form, plain;
  double ms, ms_default;
  int wino = 0;  // Winograd's form for the last level's general products
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int64_t, int64_t, uint32_t>, TuneVal> g_tune;

static bool tune_find(int64_t n, int64_t k, uint32_t p, TuneVal *v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(n, k, p));
  if (it == g_tune.end()) return false;
  *v = it->second;
  return true;
}

// Recursion depth chosen from measurements on GB300: a level pays off while
// the leaf products stay large enough to keep every SM busy at full tensor
// rate (leaf n >= 8192 at the sizes measured so far).
// Recursion depth of the untuned choice.  A level saves 1/8 of the leaves'
// ring MACs (Table 1) and costs the block additions at the HBM rate plus
// leaves with half the K, whose per-tile epilogue weighs more.  Measured with
// the BF16-digit leaf: with 3 or 4 plane products per ring MAC (p = 65521,
// 131071) no depth beats the plain lower product at n = 8192..16384,
// k = 4096..8192; with 10 (p = 2^31 - 1) one level wins at n = k = 16384.
static int auto_levels(int64_t n, int64_t k, uint32_t p) {
  const DigitSpec d = make_digits(p);
  if ((d.nsum ? d.L + d.nsum : d.L * d.L) < 6) return 0;
  int l = 0;
  while (l < 6 && (n >> (l + 1)) >= 8192 && (k >> (l + 1)) >= 2048) ++l;
  return l;
}

struct Prepared {
  int levels;
  int64_t n_pad, k_pad;
  bool padded;
};

// Recursion depth of the untuned choice for (n, k) (no AAT_LEVELS in flags).
static int prepare_levels(int64_t n, int64_t k, uint32_t p, uint32_t flags) {
  (void)p;
  const uint32_t lv = (flags & AAT_LEVELS_MASK) >> 8;
  return lv ? (int)lv - 1 : auto_levels(n, k, p);
}

static Prepared prepare(int64_t n, int64_t k, uint32_t p, const YParams &y, uint32_t flags) {
  Prepared r;
  const uint32_t lv = (flags & AAT_LEVELS_MASK) >> 8;
  r.levels = lv ? (int)lv - 1 : auto_levels(n, k, p);
  // each level halves n and k; k/2 must be even at every level for kind 2
  const int64_t mn = (int64_t)1 << r.levels;
  const int64_t mk = (int64_t)1 << (r.levels + (y.kind == 2 ? 1 : 0));
  r.n_pad = (n + mn - 1) / mn * mn;
  r.k_pad = (k + mk - 1) / mk * mk;
  if (r.levels == 0) {
    r.n_pad = n;
    r.k_pad = k;
  }
  r.padded = (r.n_pad != n || r.k_pad != k);
  return r;
}

static int validate(uint32_t p) {
  if (p >= (1u << 31)) return fail(AAT_ERANGE, "p must be below 2^31");
  if (p < 3 || (p & 1u) == 0 || !is_prime_u32(p)) return fail(AAT_ENOTPRIME, "p must be an odd prime");
  return AAT_OK;
}

static int setup(Ctx &c, uint32_t p, uint32_t flags, cudaStream_t st) {
  int e = validate(p);
  if (e) return e;
  c.m = make_modp(p);
  if (!make_y(p, &c.y)) return fail(AAT_ERANGE, "no skew-unitary Y found");
  c.ds = make_digits(p);
  if (flags & AAT_DIGITS_PLAIN) c.ds.nsum = 0;
  c.leaf = flags & AAT_LEAF_MASK;
  if (c.leaf != AAT_LEAF_TC && c.leaf != AAT_LEAF_SIMT && c.leaf != AAT_LEAF_I8 &&
      c.leaf != AAT_LEAF_F64)
    return fail(AAT_EUNSUPPORTED, "unknown leaf kind");
  // FP64 leaf: partial sums of 16 products of ((p-1)/2)^2 must stay below 2^53
  if (c.leaf == AAT_LEAF_F64 && (double)c.m.half * (double)c.m.half * 16.0 >= 9.0e15)
    return fail(AAT_ERANGE, "p too large for the exact FP64 leaf");
  const char *ew = getenv("AAT_WINOGRAD");
  c.wino = (flags & AAT_WINOGRAD) != 0 || (ew && atoi(ew) != 0);
  c.passes = (flags & AAT_LOW_MEMORY) != 0;
  c.pass_w = 1;  // set by choose_schedule
  const char *eb = getenv("AAT_EXACT_BITS");
  c.exact_bits = eb ? atoi(eb) : 24;
  c.st = st;
  c.stats = nullptr;
  return AAT_OK;
}

// Runs (or, with dry, measures) the whole product; returns workspace bytes.
// beta: null for Low(A A^T) (Table 3), else the SYRK update's beta (Table 4).
// The product (or update) on the arena as it stands (c.ar): allocations
// continue after what the caller already holds.
static size_t run_plan_in(Ctx &c, const int32_t *A, int64_t n, int64_t k, int64_t lda, int32_t *C,
                          int64_t ldc, uint32_t flags, bool dry, const MulConst *beta) {
  // choices the flags leave open come from the tuning table, if it has the shape
  TuneVal tv;
  if (c.leaf == AAT_LEAF_TC && !(flags & AAT_LEVELS_MASK) && tune_find(n, k, c.m.p, &tv)) {
    flags |= AAT_LEVELS(tv.levels);
    c.form = tv.form;
    if (tv.plain) c.ds.nsum = 0;
    if (tv.wino) c.wino = true;
  }
  Prepared pr = prepare(n, k, c.m.p, c.y, flags);
  const bool early = !pr.padded && pr.levels >= 1 && !beta && !pass_mode(c);
  // end-to-end path: with no top level to overlap, wait for all of A
  // before anything reads it
  const cudaEvent_t in_a11 = c.in_a11, in_rest = c.in_rest;
  const int nbands = c.nbands;
  if (in_rest && !early) {
    if (!dry) {
      cudaStreamWaitEvent(c.st, in_a11, 0);
      cudaStreamWaitEvent(c.st, in_rest, 0);
    }
    c.in_a11 = c.in_rest = nullptr;
    c.nbands = 0;
  }
  const int32_t *Aw = A;
  int64_t ldaw = lda;
  int32_t *Cw = C;
  int64_t ldcw = ldc;
  if (pr.padded) {
    int32_t *Ap = (int32_t *)c.ar.get((size_t)pr.n_pad * pr.k_pad * 4);
    int32_t *Cp = (int32_t *)c.ar.get((size_t)pr.n_pad * pr.n_pad * 4);
    if (!dry)
      check(c, launch_pad_copy(A, lda, n, k, Ap, pr.k_pad, pr.n_pad, pr.k_pad, c.st), "pad");
    // the SYRK update reads C: it goes into the padded copy too
    if (!dry && beta)
      check(c, launch_pad_copy(C, ldc, n, n, Cp, pr.n_pad, pr.n_pad, pr.n_pad, c.st), "pad C");
    Aw = Ap;
    ldaw = pr.k_pad;
    Cw = Cp;
    ldcw = pr.n_pad;
  }
  if (c.stats) {
    c.stats->levels = pr.levels;
    c.stats->n_pad = pr.n_pad;
    c.stats->k_pad = pr.k_pad;
  }
  c.top_levels = early ? pr.levels : -1;
  c.split_row = early ? pr.n_pad / 2 : n;

  if (beta)
    syrk_rec(c, Aw, ldaw, pr.n_pad, pr.k_pad, Cw, ldcw, pr.levels, *beta);
  else
    rec(c, Aw, ldaw, pr.n_pad, pr.k_pad, Cw, ldcw, pr.levels, no_planes());
  if (pr.padded && !dry) check(c, launch_copy_low(Cw, ldcw, C, ldc, n, c.st), "unpad");
  if (!dry && (flags & AAT_ZERO_UPPER)) check(c, launch_zero_upper(C, ldc, n, c.st), "zero upper");
  if (!dry && !early && c.split_ev && c.err == AAT_OK) cudaEventRecord(c.split_ev, c.st);
  c.in_a11 = in_a11;
  c.in_rest = in_rest;
  c.nbands = nbands;
  return c.ar.peak;
}

static size_t run_plan(Ctx &c, const int32_t *A, int64_t n, int64_t k, int64_t lda, int32_t *C,
                       int64_t ldc, uint32_t flags, bool dry, char *ws,
                       const MulConst *beta = nullptr) {
  c.ar = Arena();
  c.ar.dry = dry;
  c.ar.base = ws;
  return run_plan_in(c, A, n, k, lda, C, ldc, flags, dry, beta);
}

// The schedule of one product and its workspace (a dry run): the fast one,
// unless the flags ask for the low-memory one (AAT_LOW_MEMORY) or the fast
// one needs more than the workspace limit.  The low-memory schedule takes
// the widest plane window (fewest passes) whose workspace fits under the
// limit, or under A's own size (4 n k bytes) when no limit is set; one plane
// per pass when none fits.  AAT_PASS_PLANES (environment) fixes the width.
// Measured at n = k = 16384 over F_{2^31-1} (one level; ms, workspace):
// windows of 1, 2, 3, 4, 5, 10 planes 37.9 / 0.25 GiB, 30.7 / 0.5, 28.4 /
// 0.75, 27.9 / 1.0, 26.2 / 1.25, 25.7 / 2.5; the fast schedule 24.9 / 8.75.
static size_t choose_schedule(Ctx &c, const int32_t *A, int64_t n, int64_t k, int64_t lda,
                              int32_t *C, int64_t ldc, uint32_t flags) {
  const size_t limit = g_ws_limit.load();
  if (!c.passes) {
    const size_t need = run_plan(c, A, n, k, lda, C, ldc, flags, true, nullptr);
    if (need <= limit) return need;
    c.passes = true;
  }
  const char *epw = getenv("AAT_PASS_PLANES");
  if (epw) {
    c.pass_w = std::max(1, atoi(epw));
    return run_plan(c, A, n, k, lda, C, ldc, flags, true, nullptr);
  }
  const size_t target = limit != SIZE_MAX ? limit : (size_t)4 * (size_t)n * (size_t)k;
  size_t need = 0;
  for (int w = c.ds.L + c.ds.nsum; w >= 1; --w) {
    c.pass_w = w;
    need = run_plan(c, A, n, k, lda, C, ldc, flags, true, nullptr);
    if (need <= target) break;
  }
  return need;
}

// M M^H mod p for the quaternion matrix M = A + B i + C j + D k (Sec. 6.2,
// the 6-multiplication algorithm): U1 = A + B, U2 = C + D; five general
// products Q1 = C A^T, Q2 = D B^T, Q3 = U2 U1^T, Q4 = A B^T, Q5 = C D^T on the
// exact leaf (digit planes of A, B, C, D, U1, U2 split once and shared);
// Q6 = Low((U1 + U2)(U1 + U2)^T) by Algorithm 1 into H1; then the closing
// additions into Low(H1..H4).
static size_t quat_plan(Ctx &c, const int32_t *const M[4], int64_t n, int64_t k, int64_t lda,
                        int32_t *const H[4], int64_t ldh, uint32_t flags, bool dry, char *ws) {
  c.ar = Arena();
  c.ar.dry = dry;
  c.ar.base = ws;
  const bool tc = (c.leaf == AAT_LEAF_TC);
  int32_t *U = (int32_t *)c.ar.get((size_t)3 * n * k * 4);
  int32_t *U1 = U, *U2 = U + n * k, *U12 = U + 2 * n * k;
  int32_t *Q = (int32_t *)c.ar.get((size_t)5 * n * n * 4);
  if (!dry)
    check(c, launch_quat_sums(M[0], M[1], M[2], M[3], lda, n, k, U1, U2, U12, k, c.m, c.st),
          "quaternion sums");
  Operand o[6] = {{M[0], lda, no_planes()}, {M[1], lda, no_planes()}, {M[2], lda, no_planes()},
                  {M[3], lda, no_planes()}, {U1, k, no_planes()},   {U2, k, no_planes()}};
  if (tc)
    for (Operand &x : o) {
      x.pl = planes_alloc(c, n, k);
      if (!dry) check(c, launch_split(x.x, x.ld, n, k, c.m, c.ds.b, x.pl, c.st), "split");
    }
  const Operand &oA = o[0], &oB = o[1], &oC = o[2], &oD = o[3], &oU1 = o[4], &oU2 = o[5];
  leaf(c, oC, oA, false, n, n, k, Q + 0 * n * n, n, 0, 0);   // Q1 = C A^T
  leaf(c, oD, oB, false, n, n, k, Q + 1 * n * n, n, 0, 0);   // Q2 = D B^T
  leaf(c, oU2, oU1, false, n, n, k, Q + 2 * n * n, n, 0, 0); // Q3 = U2 U1^T
  leaf(c, oA, oB, false, n, n, k, Q + 3 * n * n, n, 0, 0);   // Q4 = A B^T
  leaf(c, oC, oD, false, n, n, k, Q + 4 * n * n, n, 0, 0);   // Q5 = C D^T
  // Q6 = Low((U1 + U2)(U1 + U2)^T) -> H1 (the tuning table may change the
  // digit form for it; the five products above keep theirs)
  const DigitSpec ds = c.ds;
  const int form = c.form;
  run_plan_in(c, U12, n, k, k, H[0], ldh, flags & ~(uint32_t)AAT_ZERO_UPPER, dry, nullptr);
  c.ds = ds;
  c.form = form;
  if (!dry) {
    check(c, launch_quat_combine(Q, n, n * n, H[0], H[1], H[2], H[3], ldh, n, c.m, c.st),
          "quaternion combine");
    if (flags & AAT_ZERO_UPPER)
      for (int q = 0; q < 4; ++q) check(c, launch_zero_upper(H[q], ldh, n, c.st), "zero upper");
  }
  return c.ar.peak;
}

static bool overlaps(const void *a, size_t an, const void *b, size_t bn) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + bn && y < x + an;
}

static int check_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3)
    return fail(AAT_ECUDA, "this library is built for sm_103a (GB300); device is sm_" +
                               std::to_string(major * 10 + minor));
  return AAT_OK;
}

// Used by the batched plans (aat_plan.cu).
int modp_levels(int64_t n, int64_t k, uint32_t p, uint32_t flags) {
  const uint32_t lv = (flags & AAT_LEVELS_MASK) >> 8;
  if (lv) return (int)lv - 1;
  TuneVal tv;
  if ((flags & AAT_LEAF_MASK) == AAT_LEAF_TC && tune_find(n, k, p, &tv)) return tv.levels;
  return auto_levels(n, k, p);
}

Planes planes_layout(const DigitSpec &ds, int64_t rows, int64_t cols) {
  return planes_for(ds, rows, cols);
}

DigitSpec digits_for_problem(int64_t n, int64_t k, uint32_t p, uint32_t flags) {
  DigitSpec d = make_digits(p);
  TuneVal tv;
  if (flags & AAT_DIGITS_PLAIN) d.nsum = 0;
  else if (!(flags & AAT_LEVELS_MASK) && (flags & AAT_LEAF_MASK) == AAT_LEAF_TC &&
           tune_find(n, k, p, &tv) && tv.plain)
    d.nsum = 0;
  return d;
}

int modp_run(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *C,
             int64_t ldc, uint32_t flags, cudaStream_t st, char *ws, bool dry, size_t *need) {
  Ctx c;
  int e = setup(c, p, flags, st);
  if (e) return e;
  // the schedule as for a single call (fast, or low-memory by flag or limit)
  size_t peak = choose_schedule(c, A, n, k, lda, C, ldc, flags);
  if (!dry) peak = run_plan(c, A, n, k, lda, C, ldc, flags, false, ws);
  if (need) *need = peak;
  return c.err;
}

// Accessors used by the allocation-free entry point (k_leaf_tc.cu).
DigitSpec digits_for_prime(uint32_t p) { return make_digits(p); }
int check_prime_arg(uint32_t p) { return validate(p); }
int check_gb300() { return check_device(); }
int report_error(int code, const char *msg) { return fail(code, msg); }
int workspace_get(size_t bytes, void **out) { return ensure_workspace(bytes, out); }

}  // namespace aat

using namespace aat;

// ================================================================ C ABI

extern "C" {

int aat_version(void) { return 100; }

const char *aat_last_error(void) { return g_last_error.c_str(); }

// aat_modp_ex with the optional early-rows event (aat_modp_host).
static int modp_device(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *C,
                       int64_t ldc, uint32_t flags, cudaStream_t stream, cudaEvent_t split_ev,
                       int64_t *split_row, int form = 0, cudaEvent_t in_a11 = nullptr,
                       cudaEvent_t in_rest = nullptr, const cudaEvent_t *in_bands = nullptr,
                       int nbands = 0) {
  if (split_row) *split_row = n;
  if (n < 0 || k < 0) return fail(AAT_EINVAL, "negative size");
  if (n > (1 << 30) || k > (1 << 30)) return fail(AAT_EINVAL, "size too large");
  if (lda < std::max<int64_t>(k, 1) || ldc < std::max<int64_t>(n, 1))
    return fail(AAT_EINVAL, "stride smaller than the row length");
  if (n > 0 && (!C || (k > 0 && !A))) return fail(AAT_EINVAL, "null pointer");
  int e;
  Ctx c;
  if ((e = setup(c, p, flags, stream))) return e;
  if (n == 0) return AAT_OK;
  if (k > 0 && overlaps(A, (size_t)((n - 1) * lda + k) * 4, C, (size_t)((n - 1) * ldc + n) * 4))
    return fail(AAT_EINVAL, "C overlaps A");
  if ((e = check_device())) return e;
  if (k == 0) {
    cudaError_t ce = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)n * 4, (size_t)n, c.st);
    return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "memset");
  }
  c.form = form;
  c.in_a11 = in_a11;
  c.in_rest = in_rest;
  c.in_bands = in_bands;
  c.nbands = in_bands ? nbands : 0;
  size_t need = choose_schedule(c, A, n, k, lda, C, ldc, flags);
  void *ws = nullptr;
  if ((e = ensure_workspace(need, &ws))) {
    // the fast schedule's workspace cannot be had: the low-memory schedule
    if (e != AAT_ENOMEM || c.passes) return e;
    c.passes = true;
    const size_t low = choose_schedule(c, A, n, k, lda, C, ldc, flags);
    if (low >= need || (e = ensure_workspace(low, &ws))) return e ? e : AAT_ENOMEM;
    g_last_error.clear();
  }
  c.err = AAT_OK;
  c.split_ev = split_ev;
  run_plan(c, A, n, k, lda, C, ldc, flags, false, (char *)ws);
  if (split_row) *split_row = c.split_row;
  return c.err;
}

// Rows [r0, r1) of the lower triangle of the n x n matrix src (device, row
// stride n) to dst (host, row stride n), in bands of kHostBand rows: band
// [a, b) copies columns [0, b) of its rows, so a band carries b (b - a)
// entries (the triangle plus (b - a)^2 / 2 entries above it).
constexpr int64_t kHostBand = 512;
// Row bands in which the end-to-end path copies A (after A11) to the device.
constexpr int kHostInBands = 8;

static int64_t low_band_entries(int64_t r0, int64_t r1) {
  int64_t total = 0;
  for (int64_t a = r0; a < r1; a += kHostBand) {
    const int64_t b = std::min(r1, a + kHostBand);
    total += b * (b - a);
  }
  return total;
}

static cudaError_t copy_low_bands(int32_t *dst, const int32_t *src, int64_t n, int64_t r0,
                                  int64_t r1, cudaStream_t st) {
  for (int64_t a = r0; a < r1; a += kHostBand) {
    const int64_t b = std::min(r1, a + kHostBand);
    cudaError_t ce = cudaMemcpy2DAsync(dst + a * n, (size_t)n * 4, src + a * n, (size_t)n * 4,
                                       (size_t)b * 4, (size_t)(b - a), cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) return ce;
  }
  return cudaSuccess;
}

int aat_modp_ex(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *C,
                int64_t ldc, uint32_t flags, void *stream) {
  g_last_error.clear();
  return modp_device(A, n, k, lda, p, C, ldc, flags, (cudaStream_t)stream, nullptr, nullptr);
}

int aat_syrk_modp(uint32_t alpha, const int32_t *A, int64_t n, int64_t k, int64_t lda,
                  uint32_t beta, int32_t *C, int64_t ldc, uint32_t p, uint32_t flags,
                  void *stream) {
  g_last_error.clear();
  if (n < 0 || k < 0) return fail(AAT_EINVAL, "negative size");
  if (n > (1 << 30) || k > (1 << 30)) return fail(AAT_EINVAL, "size too large");
  if (lda < std::max<int64_t>(k, 1) || ldc < std::max<int64_t>(n, 1))
    return fail(AAT_EINVAL, "stride smaller than the row length");
  if (n > 0 && (!C || (k > 0 && !A))) return fail(AAT_EINVAL, "null pointer");
  int e;
  Ctx c;
  if ((e = setup(c, p, flags, (cudaStream_t)stream))) return e;
  if (n == 0) return AAT_OK;
  if (k > 0 && overlaps(A, (size_t)((n - 1) * lda + k) * 4, C, (size_t)((n - 1) * ldc + n) * 4))
    return fail(AAT_EINVAL, "C overlaps A");
  if ((e = check_device())) return e;
  const MulConst b = mul_const(beta, p);
  c.alpha = mul_const(alpha, p).w;
  cudaError_t ce = cudaSuccess;
  if (k == 0 || c.alpha == 0) {
    // Low(C) <- beta Low(C)
    if (b.w == 0)
      ce = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)n * 4, (size_t)n, c.st);
    else
      ce = launch_scale_low(C, ldc, n, b, c.m, c.st);
    if (ce == cudaSuccess && (flags & AAT_ZERO_UPPER)) ce = launch_zero_upper(C, ldc, n, c.st);
    return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "scale C");
  }
  // beta = 0: the product itself (Table 3 placement), scaled by alpha
  const MulConst *pb = b.w ? &b : nullptr;
  const size_t need = run_plan(c, A, n, k, lda, C, ldc, flags, true, nullptr, pb);
  void *ws = nullptr;
  if ((e = ensure_workspace(need, &ws))) return e;
  c.err = AAT_OK;
  run_plan(c, A, n, k, lda, C, ldc, flags, false, (char *)ws, pb);
  return c.err;
}

int aah_quat_modp(const int32_t *A, const int32_t *B, const int32_t *C, const int32_t *D,
                  int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *H1, int32_t *H2,
                  int32_t *H3, int32_t *H4, int64_t ldh, uint32_t flags, void *stream) {
  g_last_error.clear();
  if (n < 0 || k < 0) return fail(AAT_EINVAL, "negative size");
  if (n > (1 << 30) || k > (1 << 30)) return fail(AAT_EINVAL, "size too large");
  if (lda < std::max<int64_t>(k, 1) || ldh < std::max<int64_t>(n, 1))
    return fail(AAT_EINVAL, "stride smaller than the row length");
  const int32_t *const M[4] = {A, B, C, D};
  int32_t *const H[4] = {H1, H2, H3, H4};
  if (n > 0) {
    for (int q = 0; q < 4; ++q)
      if (!H[q] || (k > 0 && !M[q])) return fail(AAT_EINVAL, "null pointer");
    const size_t hb = (size_t)((n - 1) * ldh + n) * 4, mb = (size_t)((n - 1) * lda + k) * 4;
    for (int q = 0; q < 4; ++q)
      for (int r = 0; r < 4; ++r) {
        if (r != q && overlaps(H[q], hb, H[r], hb)) return fail(AAT_EINVAL, "outputs overlap");
        if (k > 0 && overlaps(H[q], hb, M[r], mb)) return fail(AAT_EINVAL, "an output overlaps an input");
      }
  }
  int e;
  Ctx c;
  if ((e = setup(c, p, flags, (cudaStream_t)stream))) return e;
  if (n == 0) return AAT_OK;
  if ((e = check_device())) return e;
  if (k == 0) {
    for (int q = 0; q < 4; ++q) {
      cudaError_t ce = cudaMemset2DAsync(H[q], (size_t)ldh * 4, 0, (size_t)n * 4, (size_t)n, c.st);
      if (ce != cudaSuccess) return cuda_fail(ce, "memset");
    }
    return AAT_OK;
  }
  const size_t need = quat_plan(c, M, n, k, lda, H, ldh, flags, true, nullptr);
  void *ws = nullptr;
  if ((e = ensure_workspace(need, &ws))) return e;
  c.err = AAT_OK;
  quat_plan(c, M, n, k, lda, H, ldh, flags, false, (char *)ws);
  return c.err;
}

int aat_modp(const int32_t *A, int64_t n, int64_t k, uint32_t p, int32_t *C, void *stream) {
  return aat_modp_ex(A, n, k, k, p, C, n, 0u, stream);
}

int aat_modp_host(const int32_t *A_host, int64_t n, int64_t k, uint32_t p, int32_t *C_host,
                  uint32_t flags) {
  g_last_error.clear();
  if (n < 0 || k < 0) return fail(AAT_EINVAL, "negative size");
  if (n > 0 && (!C_host || (k > 0 && !A_host))) return fail(AAT_EINVAL, "null pointer");
  if (n == 0) return AAT_OK;
  int e;
  if ((e = check_device())) return e;
  const size_t abytes = (size_t)n * std::max<int64_t>(k, 1) * 4, cbytes = (size_t)n * n * 4;
  DeviceState *s;
  {
    std::lock_guard<std::mutex> lock(g_state_mu);
    s = &state();
    if (!s->e2e_stream) cudaStreamCreateWithFlags(&s->e2e_stream, cudaStreamNonBlocking);
    if (!s->e2e_stream2) cudaStreamCreateWithFlags(&s->e2e_stream2, cudaStreamNonBlocking);
    if (!s->e2e_split) cudaEventCreateWithFlags(&s->e2e_split, cudaEventDisableTiming);
    if (!s->e2e_a11) cudaEventCreateWithFlags(&s->e2e_a11, cudaEventDisableTiming);
    if (!s->e2e_rest) cudaEventCreateWithFlags(&s->e2e_rest, cudaEventDisableTiming);
    while ((int)s->e2e_bands.size() < kHostInBands) {
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) break;
      s->e2e_bands.push_back(ev);
    }
    if (!s->e2e_stream || !s->e2e_stream2 || !s->e2e_split || !s->e2e_a11 || !s->e2e_rest ||
        (int)s->e2e_bands.size() < kHostInBands)
      return fail(AAT_ECUDA, "e2e streams");
    if (s->e2e_a_size < abytes) {
      if (s->e2e_a) cudaFree(s->e2e_a);
      s->e2e_a = nullptr;
      s->e2e_a_size = 0;
      if (cudaMalloc(&s->e2e_a, abytes) != cudaSuccess) return fail(AAT_ENOMEM, "e2e buffer A");
      s->e2e_a_size = abytes;
    }
    if (s->e2e_c_size < cbytes) {
      if (s->e2e_c) cudaFree(s->e2e_c);
      s->e2e_c = nullptr;
      s->e2e_c_size = 0;
      if (cudaMalloc(&s->e2e_c, cbytes) != cudaSuccess) return fail(AAT_ENOMEM, "e2e buffer C");
      s->e2e_c_size = cbytes;
    }
  }
  cudaStream_t st = s->e2e_stream;
  cudaError_t ce;
  const int32_t *Cd = (const int32_t *)s->e2e_c;
  if (!(flags & AAT_ZERO_UPPER) && n >= 2 && k >= 2) {
    // A comes in on the second stream, its top-left block A11 (rows and
    // columns below n/2, k/2) first: when a recursion level runs, the
    // product P1 = Low(A11 A11^T) starts while the rest of A is in flight.
    // The rest follows in row bands (rows [i0, i1) of A12 and rows
    // [h + i0, h + i1) of the bottom half), so that the top level's S-block
    // kernel, which needs the rows i and h + i of all four blocks, runs on
    // each band as soon as it is on the device.
    int32_t *Ad = (int32_t *)s->e2e_a;
    const int64_t h = n / 2, kap = k / 2;
    cudaStream_t s2 = s->e2e_stream2;
    if ((ce = cudaMemcpy2DAsync(Ad, (size_t)k * 4, A_host, (size_t)k * 4, (size_t)kap * 4,
                                (size_t)h, cudaMemcpyHostToDevice, s2)) != cudaSuccess ||
        (ce = cudaEventRecord(s->e2e_a11, s2)) != cudaSuccess)
      return cuda_fail(ce, "copy A to the device");
    for (int b = 0; b < kHostInBands; ++b) {
      const int64_t i0 = h * b / kHostInBands, i1 = h * (b + 1) / kHostInBands;
      // the last band also carries the bottom row of an odd n
      const int64_t j1 = (b == kHostInBands - 1) ? n : h + i1;
      if (i1 > i0 && (ce = cudaMemcpy2DAsync(Ad + i0 * k + kap, (size_t)k * 4,
                                             A_host + i0 * k + kap, (size_t)k * 4,
                                             (size_t)(k - kap) * 4, (size_t)(i1 - i0),
                                             cudaMemcpyHostToDevice, s2)) != cudaSuccess)
        return cuda_fail(ce, "copy A to the device");
      if (j1 > h + i0 && (ce = cudaMemcpyAsync(Ad + (h + i0) * k, A_host + (h + i0) * k,
                                               (size_t)(j1 - h - i0) * k * 4,
                                               cudaMemcpyHostToDevice, s2)) != cudaSuccess)
        return cuda_fail(ce, "copy A to the device");
      if ((ce = cudaEventRecord(s->e2e_bands[b], s2)) != cudaSuccess)
        return cuda_fail(ce, "copy A to the device");
    }
    if ((ce = cudaEventRecord(s->e2e_rest, s2)) != cudaSuccess)
      return cuda_fail(ce, "copy A to the device");
    // only the lower triangle is defined: copy it in row bands; the rows
    // below the top-level split are final before the last product P2 runs
    // and go back on the second stream meanwhile
    int64_t split = n;
    e = modp_device(Ad, n, k, k, p, (int32_t *)Cd, n, flags, st, s->e2e_split, &split, 0,
                    s->e2e_a11, s->e2e_rest, s->e2e_bands.data(), kHostInBands);
    if (e) return e;
    if (split < n) {
      if ((ce = cudaStreamWaitEvent(s2, s->e2e_split, 0)) != cudaSuccess ||
          (ce = copy_low_bands(C_host, Cd, n, split, n, s2)) != cudaSuccess)
        return cuda_fail(ce, "copy C to the host");
    }
    if ((ce = copy_low_bands(C_host, Cd, n, 0, split, st)) != cudaSuccess)
      return cuda_fail(ce, "copy C to the host");
    if ((ce = cudaStreamSynchronize(s2)) != cudaSuccess) return cuda_fail(ce, "synchronize");
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ce, "synchronize");
    return AAT_OK;
  }
  if (k > 0 && (ce = cudaMemcpyAsync(s->e2e_a, A_host, (size_t)n * k * 4, cudaMemcpyHostToDevice,
                                     st)) != cudaSuccess)
    return cuda_fail(ce, "copy A to the device");
  if (flags & AAT_ZERO_UPPER) {
    // the caller asked for the whole matrix: one copy at the end
    e = modp_device((const int32_t *)s->e2e_a, n, k, std::max<int64_t>(k, 1), p, (int32_t *)Cd, n,
                    flags, st, nullptr, nullptr);
    if (e) return e;
    if ((ce = cudaMemcpyAsync(C_host, Cd, cbytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(ce, "copy C to the host");
  } else {
    // only the lower triangle is defined: copy it in row bands; the rows
    // below the top-level split are final before the last product P2 runs
    // and go back on a second stream meanwhile
    int64_t split = n;
    e = modp_device((const int32_t *)s->e2e_a, n, k, std::max<int64_t>(k, 1), p, (int32_t *)Cd, n,
                    flags, st, s->e2e_split, &split);
    if (e) return e;
    if (split < n) {
      if ((ce = cudaStreamWaitEvent(s->e2e_stream2, s->e2e_split, 0)) != cudaSuccess ||
          (ce = copy_low_bands(C_host, Cd, n, split, n, s->e2e_stream2)) != cudaSuccess)
        return cuda_fail(ce, "copy C to the host");
    }
    if ((ce = copy_low_bands(C_host, Cd, n, 0, split, st)) != cudaSuccess)
      return cuda_fail(ce, "copy C to the host");
    if ((ce = cudaStreamSynchronize(s->e2e_stream2)) != cudaSuccess)
      return cuda_fail(ce, "synchronize");
  }
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ce, "synchronize");
  return AAT_OK;
}

int aat_tune_modp(int64_t n, int64_t k, uint32_t p, uint32_t flags, int reps, void *stream,
                  aat_tune_t *out) {
  g_last_error.clear();
  if (!out) return fail(AAT_EINVAL, "null pointer");
  if (n <= 0 || k <= 0 || n > (1 << 30) || k > (1 << 30)) return fail(AAT_EINVAL, "bad size");
  if ((flags & AAT_LEAF_MASK) != AAT_LEAF_TC)
    return fail(AAT_EUNSUPPORTED, "tuning covers the tensor-core leaf");
  // the tuned choices themselves are not flags of the candidates
  flags &= ~(AAT_LEVELS_MASK | AAT_DIGITS_PLAIN | AAT_WINOGRAD | AAT_ZERO_UPPER);
  cudaStream_t st = (cudaStream_t)stream;
  int e;
  {
    Ctx c0;
    if ((e = setup(c0, p, flags, st))) return e;
  }
  if ((e = check_device())) return e;
  reps = std::min(std::max(reps, 1), 50);
  int32_t *A = nullptr, *C = nullptr;
  if (cudaMalloc(&A, (size_t)n * k * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(AAT_ENOMEM, "tuning input");
  }
  if (cudaMalloc(&C, (size_t)n * n * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(A);
    return fail(AAT_ENOMEM, "tuning output");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t ce = launch_fill_residues(A, n * k, p, 0x2101010250ull, st);
  // candidates: the untuned choice first, then every (levels, form, digits)
  struct Cand {
    uint32_t flags;
    int levels, form, plain;
    double ms;
    int wino;
  };
  std::vector<Cand> cands;
  cands.push_back({flags, -1, 0, 0, 1e300, 0});
  int maxl = 0;
  while (maxl < 3 && (n >> (maxl + 1)) >= 512 && (k >> (maxl + 1)) >= 128) ++maxl;
  const bool sums = make_digits(p).nsum > 0;
  for (int l = 0; l <= maxl; ++l)
    for (int form = 1; form <= 2; ++form) {
      if (form == 2 && (n >> l) < 256) continue;  // no leaf tall enough for a pair
      for (int plain = 0; plain <= (sums ? 1 : 0); ++plain)
        cands.push_back({flags | AAT_LEVELS(l) | (plain ? AAT_DIGITS_PLAIN : 0u), l, form, plain,
                         1e300, 0});
      // Winograd's form for the last level's general products (default digits)
      if (l >= 1)
        cands.push_back({flags | AAT_LEVELS(l) | AAT_WINOGRAD, l, form, 0, 1e300, 1});
    }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.erase(std::make_tuple(n, k, p));
  }
  if (ce != cudaSuccess) e = cuda_fail(ce, "tuning input");
  // one untimed run of each, then `reps` rounds that time every candidate
  // once, round robin (clock and power drift spread evenly); best of rounds
  for (size_t i = 0; i < cands.size() && !e; ++i)
    e = modp_device(A, n, k, k, p, C, n, cands[i].flags, st, nullptr, nullptr, cands[i].form);
  for (int r = 0; r < reps && !e; ++r)
    for (size_t i = 0; i < cands.size() && !e; ++i) {
      cudaEventRecord(e0, st);
      e = modp_device(A, n, k, k, p, C, n, cands[i].flags, st, nullptr, nullptr, cands[i].form);
      cudaEventRecord(e1, st);
      cudaError_t se = cudaEventSynchronize(e1);
      if (!e && se != cudaSuccess) e = cuda_fail(se, "tuning run");
      float t = 0.f;
      if (!e) cudaEventElapsedTime(&t, e0, e1);
      cands[i].ms = std::min(cands[i].ms, (double)t);
    }
  // the fastest, unless it beats the untuned choice by less than 2 %
  size_t bi = 1;
  for (size_t i = 1; i < cands.size(); ++i)
    if (cands[i].ms < cands[bi].ms) bi = i;
  const double ms_default = cands[0].ms;
  TuneVal best;
  if (cands.size() < 2 || cands[bi].ms > 0.98 * ms_default)
    best = TuneVal{prepare_levels(n, k, p, flags), 0, 0, ms_default, 0.0};
  else
    best = TuneVal{cands[bi].levels, cands[bi].form, cands[bi].plain, cands[bi].ms, 0.0,
                   cands[bi].wino};
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(A);
  cudaFree(C);
  if (e) return e;
  best.ms_default = ms_default;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[std::make_tuple(n, k, p)] = best;
  }
  out->levels = best.levels;
  out->form = best.form;
  out->plain_digits = best.plain;
  out->winograd = best.wino;
  out->ms = best.ms;
  out->ms_default = best.ms_default;
  return AAT_OK;
}

int aat_tune_lookup(int64_t n, int64_t k, uint32_t p, aat_tune_t *out) {
  TuneVal v;
  if (!tune_find(n, k, p, &v)) return 0;
  if (out) {
    out->levels = v.levels;
    out->form = v.form;
    out->plain_digits = v.plain;
    out->winograd = v.wino;
    out->ms = v.ms;
    out->ms_default = v.ms_default;
  }
  return 1;
}

void aat_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
}

static std::string device_name() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return std::string();
  }
  std::string name(prop.name);
  for (char &ch : name)
    if (ch == '"' || ch == '\\' || ch < 32) ch = ' ';
  return name;
}

int aat_tune_save(const char *path) {
  g_last_error.clear();
  if (!path) return fail(AAT_EINVAL, "null path");
  FILE *f = fopen(path, "w");
  if (!f) return fail(AAT_EINVAL, std::string("cannot write ") + path);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  fprintf(f, "{\"gpu\": \"%s\", \"entries\": [\n", device_name().c_str());
  size_t i = 0;
  for (const auto &kv : g_tune) {
    const TuneVal &v = kv.second;
    fprintf(f,
            "  {\"n\": %lld, \"k\": %lld, \"p\": %u, \"levels\": %d, \"form\": %d, "
            "\"plain_digits\": %d, \"ms\": %.6f, \"ms_default\": %.6f, \"winograd\": %d}%s\n",
            (long long)std::get<0>(kv.first), (long long)std::get<1>(kv.first),
            (unsigned)std::get<2>(kv.first), v.levels, v.form, v.plain, v.ms, v.ms_default,
            v.wino, ++i < g_tune.size() ? "," : "");
  }
  fprintf(f, "]}\n");
  const bool ok = (fclose(f) == 0);
  if (!ok) return fail(AAT_EINVAL, std::string("cannot write ") + path);
  return (int)g_tune.size();
}

int aat_tune_load(const char *path) {
  g_last_error.clear();
  if (!path) return fail(AAT_EINVAL, "null path");
  FILE *f = fopen(path, "r");
  if (!f) return fail(AAT_EINVAL, std::string("cannot read ") + path);
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  fclose(f);
  // entries tuned on another kind of GPU do not apply here
  const std::string here = device_name();
  const size_t g = text.find("\"gpu\": \"");
  if (g != std::string::npos && !here.empty()) {
    const size_t b = g + 8, q = text.find('"', b);
    if (q == std::string::npos || text.compare(b, q - b, here) != 0) return 0;
  }
  int count = 0;
  size_t pos = 0;
  while ((pos = text.find("{\"n\":", pos)) != std::string::npos) {
    long long n = 0, k = 0;
    unsigned p = 0;
    int levels = -1, form = -1, plain = -1, wino = 0;
    double ms = 0.0, msd = 0.0;
    // "winograd" is optional (files written before it was tuned lack it)
    const int m = sscanf(text.c_str() + pos,
                         "{\"n\": %lld, \"k\": %lld, \"p\": %u, \"levels\": %d, \"form\": %d, "
                         "\"plain_digits\": %d, \"ms\": %lf, \"ms_default\": %lf, "
                         "\"winograd\": %d}",
                         &n, &k, &p, &levels, &form, &plain, &ms, &msd, &wino);
    ++pos;
    if (m < 8 || n <= 0 || k <= 0 || n > (1 << 30) || k > (1 << 30) || levels < 0 ||
        levels > 14 || form < 0 || form > 2 || (plain != 0 && plain != 1) ||
        (wino != 0 && wino != 1) || validate(p) != AAT_OK)
      continue;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[std::make_tuple((int64_t)n, (int64_t)k, (uint32_t)p)] =
        TuneVal{levels, form, plain, ms, msd, wino};
    ++count;
  }
  g_last_error.clear();
  return count;
}

int64_t aat_modp_host_d2h_bytes(int64_t n, uint32_t flags) {
  if (n <= 0) return 0;
  if (flags & AAT_ZERO_UPPER) return n * n * 4;
  return 4 * low_band_entries(0, n);
}

int aat_gemm_modp(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy, int64_t m,
                  int64_t n, int64_t k, uint32_t p, int32_t *C, int64_t ldc, uint32_t flags,
                  void *stream) {
  g_last_error.clear();
  if (m < 0 || n < 0 || k < 0) return fail(AAT_EINVAL, "negative size");
  if (ldx < std::max<int64_t>(k, 1) || ldy < std::max<int64_t>(k, 1) ||
      ldc < std::max<int64_t>(n, 1))
    return fail(AAT_EINVAL, "stride smaller than the row length");
  if (m > 0 && n > 0 && (!C || (k > 0 && (!X || !Y)))) return fail(AAT_EINVAL, "null pointer");
  int e;
  Ctx c;
  if ((e = setup(c, p, flags, (cudaStream_t)stream))) return e;
  if (m == 0 || n == 0) return AAT_OK;
  if ((e = check_device())) return e;
  if (k == 0) {
    cudaError_t ce = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)n * 4, (size_t)m, c.st);
    return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "memset");
  }
  const bool same = (X == Y && ldx == ldy && m == n);
  size_t need = 0;
  for (int pass = 0; pass < 2; ++pass) {
    void *ws = nullptr;
    c.ar = Arena();
    c.ar.dry = (pass == 0);
    if (pass == 1) {
      if ((e = ensure_workspace(need, &ws))) return e;
      c.ar.base = (char *)ws;
    }
    Operand ox{X, ldx, no_planes()}, oy{Y, ldy, no_planes()};
    leaf(c, ox, oy, same, m, n, k, C, ldc, 0, 0);
    need = c.ar.peak;
  }
  return c.err;
}

size_t aat_workspace_size(int64_t n, int64_t k, uint32_t p, uint32_t flags) {
  Ctx c;
  if (n <= 0 || k <= 0 || setup(c, p, flags, nullptr)) return 0;
  return choose_schedule(c, nullptr, n, k, k, nullptr, n, flags);
}

void aat_set_workspace_limit(size_t bytes) { g_ws_limit.store(bytes); }

int aat_device_status(int reset) {
  int32_t *d = device_status_ptr();
  if (!d) return fail(AAT_ECUDA, "no device status word");
  cudaError_t ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) return cuda_fail(ce, "synchronize");
  int32_t v = 0;
  cudaMemcpy(&v, d, sizeof(v), cudaMemcpyDeviceToHost);
  if (reset) cudaMemset(d, 0, sizeof(int32_t));
  // the allocation-free entry point keeps its own word in its static array
  const int w = noalloc_status(reset);
  return v != AAT_OK ? v : w;
}

void aat_shutdown(void) {
  cudaDeviceSynchronize();
  leaf_tc_release();
  leaf_f32_release();
  std::lock_guard<std::mutex> lock(g_state_mu);
  for (auto &kv : g_states) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first);
    DeviceState &s = kv.second;
    if (s.ws) cudaFree(s.ws);
    if (s.status) cudaFree(s.status);
    if (s.e2e_a) cudaFree(s.e2e_a);
    if (s.e2e_c) cudaFree(s.e2e_c);
    if (s.e2e_stream) cudaStreamDestroy(s.e2e_stream);
    if (s.e2e_stream2) cudaStreamDestroy(s.e2e_stream2);
    if (s.e2e_split) cudaEventDestroy(s.e2e_split);
    if (s.e2e_a11) cudaEventDestroy(s.e2e_a11);
    if (s.e2e_rest) cudaEventDestroy(s.e2e_rest);
    for (cudaEvent_t ev : s.e2e_bands) cudaEventDestroy(ev);
    cudaSetDevice(cur);
  }
  g_states.clear();
}

int aat_profile_begin(void) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  for (auto &r : g_prof) {
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.clear();
  g_prof_on = true;
  return AAT_OK;
}

int aat_profile_end(aat_profile_t *out) {
  cudaError_t ce = cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_prof_on = false;
  if (out) std::memset(out, 0, sizeof(*out));
  for (auto &r : g_prof) {
    float ms = 0.f;
    if (ce == cudaSuccess && out && r.cls >= 0 && r.cls < AAT_K_NCLASS &&
        cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      out->launches[r.cls] += 1;
      out->ms[r.cls] += ms;
      out->work[r.cls] += r.work;
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.clear();
  return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "profile synchronize");
}

// ------------------------------------------------------------ test hooks

int aatx_is_prime(uint64_t p) { return is_prime_u32(p) ? 1 : 0; }

int64_t aatx_sqrt_mod(int64_t a, uint64_t p) {
  uint64_t r;
  if (p < 3 || !is_prime_u32(p)) return -1;
  return sqrt_mod(canon64(a, p), p, &r) ? (int64_t)r : -1;
}

int aatx_sos(int64_t k, uint64_t p, uint64_t *a, uint64_t *b) {
  if (p < 3 || !is_prime_u32(p)) return AAT_ENOTPRIME;
  return sos(canon64(k, p), p, a, b) ? AAT_OK : AAT_ERANGE;
}

int aatx_y_params(uint32_t p, int *kind, uint32_t *a, uint32_t *b) {
  int e = validate(p);
  if (e) return e;
  YParams y;
  if (!make_y(p, &y)) return fail(AAT_ERANGE, "no Y");
  *kind = y.kind;
  *a = (uint32_t)(y.a < 0 ? y.a + (int64_t)p : y.a);
  *b = (uint32_t)(y.b < 0 ? y.b + (int64_t)p : y.b);
  return AAT_OK;
}

int aatx_digit_spec(uint32_t p, int *b, int *L, int *dmax, int *nsum) {
  int e = validate(p);
  if (e) return e;
  DigitSpec d = make_digits(p);
  *b = d.b;
  *L = d.L;
  for (int i = 0; i < 8; ++i) dmax[i] = d.dmax[i];
  *nsum = d.nsum;
  return AAT_OK;
}

int aatx_plan_stats(int64_t n, int64_t k, uint32_t p, uint32_t flags, aatx_plan_stats_t *out) {
  if (!out || n <= 0 || k <= 0) return fail(AAT_EINVAL, "bad arguments");
  std::memset(out, 0, sizeof(*out));
  Ctx c;
  int e = setup(c, p, flags, nullptr);
  if (e) return e;
  c.stats = out;
  out->workspace_bytes = run_plan(c, nullptr, n, k, k, nullptr, n, flags, true, nullptr);
  return AAT_OK;
}

int aatx_sblocks(const int32_t *A, int64_t n, int64_t k, int64_t lda, uint32_t p, int32_t *S1,
                 int32_t *S2, int32_t *S3, int32_t *S4, int64_t lds, void *stream) {
  Ctx c;
  int e = setup(c, p, 0, (cudaStream_t)stream);
  if (e) return e;
  if ((e = check_device())) return e;
  if (n % 2 || k % 2 || (c.y.kind == 2 && (k / 2) % 2)) return fail(AAT_EINVAL, "bad shape");
  SKernelOut o;
  std::memset(&o, 0, sizeof(o));
  int32_t *S[4] = {S1, S2, S3, S4};
  for (int q = 0; q < 4; ++q) {
    o.s[q] = S[q];
    o.lds[q] = lds;
  }
  cudaError_t ce = launch_sblocks(A, lda, n / 2, k / 2, c.m, c.y, c.ds.b, o, c.st);
  return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "sblocks");
}

int aatx_split(const int32_t *X, int64_t rows, int64_t cols, int64_t ldx, uint32_t p,
               uint16_t *planes, void *stream) {
  Ctx c;
  int e = setup(c, p, 0, (cudaStream_t)stream);
  if (e) return e;
  if ((e = check_device())) return e;
  Planes P = planes_for(c.ds, rows, cols);
  P.ptr = (__nv_bfloat16 *)planes;
  cudaError_t ce = launch_split(X, ldx, rows, cols, c.m, c.ds.b, P, c.st);
  return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "split");
}

int aatx_leaf(const int32_t *X, int64_t ldx, const int32_t *Y, int64_t ldy, int64_t M, int64_t N,
              int64_t K, uint32_t p, int32_t *C, int64_t ldc, int lower, int accumulate,
              uint32_t leafkind, int exact_bits, void *stream) {
  Ctx c;
  int e = setup(c, p, leafkind, (cudaStream_t)stream);
  if (e) return e;
  if ((e = check_device())) return e;
  if (exact_bits > 0) c.exact_bits = exact_bits;
  if (M <= 0 || N <= 0 || K <= 0) return fail(AAT_EINVAL, "bad sizes");
  const bool same = (X == Y && ldx == ldy && M == N);
  size_t need = 0;
  for (int pass = 0; pass < 2; ++pass) {
    void *ws = nullptr;
    c.ar = Arena();
    c.ar.dry = (pass == 0);
    if (pass == 1) {
      if ((e = ensure_workspace(need, &ws))) return e;
      c.ar.base = (char *)ws;
    }
    Operand ox{X, ldx, no_planes()}, oy{Y, ldy, no_planes()};
    leaf(c, ox, oy, same, M, N, K, C, ldc, lower, accumulate);
    need = c.ar.peak;
  }
  return c.err;
}

void aatx_set_alloc_limit(size_t bytes) { g_alloc_limit.store(bytes); }

int aatx_workspace_reserve(size_t bytes) {
  void *ws = nullptr;
  return ensure_workspace(bytes, &ws);
}

int aatx_postadd(int32_t *C, int64_t ldc, int64_t h, uint32_t p, void *stream) {
  Ctx c;
  int e = setup(c, p, 0, (cudaStream_t)stream);
  if (e) return e;
  if ((e = check_device())) return e;
  cudaError_t ce =
      launch_postadd(C, ldc, C + h, C + h * ldc, C + h * ldc + h, ldc, h, c.m, (cudaStream_t)stream);
  return ce == cudaSuccess ? AAT_OK : cuda_fail(ce, "postadd");
}

}  // extern "C"
