// common.cuh — shared definitions of the NUMARCK sm_103a kernels.
//
// Method arithmetic follows the paper's compression steps (arXiv 1703.02438: Eq. 1 change
// ratio, §IV.B.1 top-k binning, §III.C indexing, Eq. 4 reconstruction) in the element type T,
// round-to-nearest-even, no fused multiply-add (the library is built with -fmad=false and every
// method operation below is an explicit _rn intrinsic).
//
// GB300's FP64 pipe issues about 0.5 T ops/s, far below what HBM delivers per element, so the
// float64 bin and error-bound decisions run a float32 estimate with a proven error bound first
// and only fall back to the exact float64 sequence when the estimate cannot decide (the
// result is identical to the exact sequence by construction; see classify_f64 / check_f64).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "numarck.h"

namespace nmk {

constexpr int SUB = NUMARCK_SUB_BLOCK;          // elements per sub-block (= K3/K4 tile)
constexpr int WIN_LOG2 = NUMARCK_WINDOW_LOG2;   // |ratio| <= 2^21 * w
constexpr int HWIN = (1 << (WIN_LOG2 + 1)) + 16; // global histogram window (bins)
constexpr int HMARGIN = 8;                      // spare bins at each end of the window
constexpr int SH_BINS = 16384;                  // K1 shared-memory histogram window
constexpr int DM_SMEM = 4096;                   // K4 multipliers kept in shared memory
constexpr unsigned KEY_BIAS = 0x40000000u;      // bin-range keys: 0 means "no value"
constexpr int SCAN_TILE = 4096;                 // per-tile counts one offset-scan CTA covers
// Per-element codes written by K1 and read by K3. For a binnable point whose bin b lies in the
// code window [code_base, code_base + CODE_BINS) (code_base = zero-change bin - 16383):
// code = (b - code_base) << 1 | pass, where pass is the error-bound check of §III.C against the
// centre of b itself (the only centre a point can be indexed to). CODE_FAR marks binnable points
// outside the window (K3 classifies and checks them again from prev and cur), CODE_NONE points
// that are not binnable. CODE_NONE is even (pass bit clear) and CODE_FAR odd, and both have
// code >> 1 = CODE_BINS, one past the last bin of the window.
constexpr unsigned CODE_NONE = 0xFFFEu;
constexpr unsigned CODE_FAR = 0xFFFFu;
constexpr int CODE_BINS = 32767;
constexpr int CODE_HALF = 16383;

// Workspace control block (first 256 bytes of the workspace). Zero at entry of every
// compression; the kernels restore the zero state of every field they accumulate into.
struct Ctrl {
  unsigned int bmin_key;        // max over binnable points of (KEY_BIAS - bin)
  unsigned int bmax_key;        // max over binnable points of (bin + KEY_BIAS)
  unsigned long long amin_key;  // ANCHOR_MIN: max of ~orderable(ratio)
  unsigned int ticket;          // order of the offset-scan CTAs (reset by K1)
  int error;                    // device-side NUMARCK_ERR_* of the current call
  // written by K2 for K3 (plain stores; no reset needed)
  int any;                      // 1 if at least one point is binnable
  int sel_bmin, sel_bmax;       // bin range of the binnable points
  int n_sel;                    // selected bins
  int pad0;
  double a;                     // grid anchor (the T value, widened)
  unsigned int win_err;         // a bin fell outside the histogram window (never expected)
  int code_base;                // bin of code 0 in K1's per-point codes (written by K1)
  int sel_lo, sel_hi;           // bin range of the selected bins (sel_lo > sel_hi: none)
  int auto_B;                   // index length chosen from the histogram (B = 0 requests)
  unsigned int pad1[45];
};
static_assert(sizeof(Ctrl) == 256, "Ctrl must be 256 bytes");

// Byte offsets of the workspace regions (computed on the host).
struct WsLayout {
  size_t ctrl, hist, rank, mtab, cftab, selb, status, total;
};

// Blob geometry (computed on the host from n and the parameters).
struct Geometry {
  int64_t n, epb, nblocks, nsub, spb, block_stride, index_bytes;
  int64_t off_centres, off_idx_off, off_inc_off, off_sub_off, off_index, off_exact;
  int B;
  int M;          // marker = 2^B - 1
  int dtype;
  int anchor;
};

__host__ __device__ __forceinline__ int64_t round_up_i64(int64_t x, int64_t m) {
  return (x + m - 1) / m * m;
}
__host__ __device__ __forceinline__ int64_t ceil_div_i64(int64_t a, int64_t b) {
  return (a + b - 1) / b;
}

// Blob geometry of the documented format (§IV.C block layout, §IV.D arrays, Fig. 2): a pure
// function of (n, dtype, B, block_bytes). Used to build headers and to validate them.
__host__ __device__ inline Geometry make_geometry(int64_t n, int dtype, int B, int64_t block_bytes,
                                                  int anchor) {
  Geometry g{};
  const int64_t L = dtype == NUMARCK_F64 ? 8 : 4;
  g.n = n;
  g.B = B;
  g.M = (1 << B) - 1;
  g.dtype = dtype;
  g.anchor = anchor;
  g.epb = (8 * block_bytes) / B;
  g.nblocks = n > 0 ? ceil_div_i64(n, g.epb) : 0;
  g.spb = ceil_div_i64(g.epb, SUB);
  const int64_t last = g.nblocks ? n - (g.nblocks - 1) * g.epb : 0;
  g.nsub = g.nblocks ? (g.nblocks - 1) * g.spb + ceil_div_i64(last, SUB) : 0;
  g.block_stride = round_up_i64(ceil_div_i64(g.epb * B, 8), 16);
  g.index_bytes =
      g.nblocks ? (g.nblocks - 1) * g.block_stride + round_up_i64(ceil_div_i64(last * B, 8), 16) : 0;
  g.off_centres = NUMARCK_HEADER_BYTES;
  g.off_idx_off = round_up_i64(g.off_centres + ((int64_t)1 << B) * L, NUMARCK_SECTION_ALIGN);
  g.off_inc_off = round_up_i64(g.off_idx_off + (g.nblocks + 1) * 8, NUMARCK_SECTION_ALIGN);
  g.off_sub_off = round_up_i64(g.off_inc_off + (g.nblocks + 1) * 8, NUMARCK_SECTION_ALIGN);
  g.off_index = round_up_i64(g.off_sub_off + g.nsub * 8, NUMARCK_SECTION_ALIGN);
  g.off_exact = round_up_i64(g.off_index + g.index_bytes, NUMARCK_SECTION_ALIGN);
  return g;
}

constexpr int64_t MAX_N = (int64_t)1 << 40;

// Byte offset of K1's per-element codes inside the blob buffer: the tail of the
// incompressible-value capacity, rounded down to 16 bytes (element j at + 2j). K3a consumes a
// tile's codes before anything is written over them (its own marker ballots); K3c reads those
// ballots only while the incompressible table ends at or below this offset.
__host__ __device__ __forceinline__ int64_t code_offset(const Geometry& g) {
  return (g.off_exact + g.n * ((g.dtype == NUMARCK_F64 ? 8 : 4) - 2)) & ~(int64_t)15;
}

// The header of a compression as known before its kernels run (status, n_sel, n_inc and a are
// 0; the kernels fill them in): magic, version, parameters and the section offsets of g.
__host__ __device__ inline numarck_header make_header(const Geometry& g, double E,
                                                      int64_t block_bytes) {
  numarck_header h;
  unsigned char* raw = reinterpret_cast<unsigned char*>(&h);
  for (int i = 0; i < (int)sizeof(h); ++i) raw[i] = 0;
  h.magic = NUMARCK_MAGIC;
  h.version = NUMARCK_VERSION;
  h.dtype = g.dtype;
  h.B = g.B;
  h.E = E;
  h.anchor = g.anchor;
  h.n = g.n;
  h.block_bytes = block_bytes;
  h.epb = g.epb;
  h.nblocks = g.nblocks;
  h.sub = SUB;
  h.nsub = g.nsub;
  h.block_stride = g.block_stride;
  h.off_centres = g.off_centres;
  h.off_idx_off = g.off_idx_off;
  h.off_inc_off = g.off_inc_off;
  h.off_sub_off = g.off_sub_off;
  h.off_index = g.off_index;
  h.off_exact = g.off_exact;
  h.total_bytes = g.off_exact;
  return h;
}

// Checks a header against the geometry its own fields imply. Returns 0 or NUMARCK_ERR_CORRUPT
// (or the header's non-zero device status).
__host__ __device__ inline int check_header(const numarck_header& h, Geometry* out) {
  if (h.magic != NUMARCK_MAGIC || h.version != NUMARCK_VERSION) return NUMARCK_ERR_CORRUPT;
  if (h.status != 0) return h.status;
  if (h.dtype != NUMARCK_F32 && h.dtype != NUMARCK_F64) return NUMARCK_ERR_CORRUPT;
  if (h.B < 1 || h.B > NUMARCK_MAX_B) return NUMARCK_ERR_CORRUPT;
  if (h.anchor != NUMARCK_ANCHOR_ZERO && h.anchor != NUMARCK_ANCHOR_MIN) return NUMARCK_ERR_CORRUPT;
  if (h.n < 0 || h.n > MAX_N) return NUMARCK_ERR_CORRUPT;
  if (h.block_bytes < 2 || h.block_bytes > ((int64_t)1 << 30)) return NUMARCK_ERR_CORRUPT;
  if (h.sub != SUB) return NUMARCK_ERR_CORRUPT;
  const Geometry g = make_geometry(h.n, h.dtype, h.B, h.block_bytes, h.anchor);
  if (h.epb != g.epb || h.nblocks != g.nblocks || h.nsub != g.nsub ||
      h.block_stride != g.block_stride || h.off_centres != g.off_centres ||
      h.off_idx_off != g.off_idx_off || h.off_inc_off != g.off_inc_off ||
      h.off_sub_off != g.off_sub_off || h.off_index != g.off_index || h.off_exact != g.off_exact)
    return NUMARCK_ERR_CORRUPT;
  if (h.n_sel < 0 || h.n_sel > g.M || h.n_inc < 0 || h.n_inc > h.n) return NUMARCK_ERR_CORRUPT;
  const int64_t L = h.dtype == NUMARCK_F64 ? 8 : 4;
  if (h.total_bytes != g.off_exact + h.n_inc * L) return NUMARCK_ERR_CORRUPT;
  if (out) *out = g;
  return 0;
}

// Constants of the T-precision chain plus the float32 estimate constants (float64 only).
template <typename T>
struct Consts {
  T E_T, w, inv_w, cap, a;
  int hbase;      // histogram window index = bin - hbase
  // float64 estimate: af = fl32(a), inv_wf = fl32(inv_w), Ef = fl32(E_T), wf = fl32(w),
  // cap_lo <= min(cap (1 - 2^-19), 2^100), cap_hi >= cap (1 + 2^-19),
  // K0 >= 2^-19 inv_w |a| + 2^-60, and for K1's own-bin check kA >= 2^-22 + 2^-23 + 2^-50,
  // k1 >= 2^-20 (1 + Ef), C0 >= 2^-22 |af| + 2^-49 + 2^-50 + 2^-100 (all rounded away from
  // the decision)
  float af, inv_wf, Ef, cap_lo, cap_hi, K0, wf, kA, k1, C0;
};

// ------------------------------------------------------------------------------------------
// small device helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
// Waits until ready(*p) holds (relaxed loads at GPU scope, backing off with nanosleep once 64
// polls have failed), for at most limit_ns of the global timer from then on. Returns true with
// the value in v, or false when the limit expires: every wait of a kernel on another CTA is
// bounded this way, so a flag that is never set becomes an error status instead of a hang.
template <typename Ready>
__device__ __forceinline__ bool bounded_wait(const unsigned long long* p,
                                             unsigned long long limit_ns, unsigned long long& v,
                                             Ready ready) {
  unsigned spins = 0;
  unsigned long long t0 = 0;
  for (;;) {
    v = ld_relaxed_u64(p);
    if (ready(v)) return true;
    if (++spins == 64) t0 = global_timer_ns();
    if (spins > 64) {
      __nanosleep(100);
      if ((spins & 63u) == 0 && global_timer_ns() - t0 > limit_ns) return false;
    }
  }
}

// 16-byte asynchronous copies global -> shared (cp.async, bypassing L1), committed as a group.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n"
               :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Index v of the variable whose range [pre[v], pre[v+1]) holds x, for a non-decreasing prefix
// table pre[0..count] with pre[0] = 0 <= x < pre[count] (variables with empty ranges are
// skipped: the largest v with pre[v] <= x).
__device__ __forceinline__ int find_var(const long long* pre, int count, long long x) {
  int lo = 0, hi = count;          // pre[lo] <= x < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Streaming loads (read once, do not keep in L1).
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }

// T-precision round-to-nearest operations (explicit, never contracted).
__device__ __forceinline__ float  t_sub(float a, float b)   { return __fsub_rn(a, b); }
__device__ __forceinline__ double t_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float  t_add(float a, float b)   { return __fadd_rn(a, b); }
__device__ __forceinline__ double t_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float  t_mul(float a, float b)   { return __fmul_rn(a, b); }
__device__ __forceinline__ double t_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float  t_div(float a, float b)   { return __fdiv_rn(a, b); }
__device__ __forceinline__ double t_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float  t_abs(float a)  { return fabsf(a); }
__device__ __forceinline__ double t_abs(double a) { return fabs(a); }
__device__ __forceinline__ float  t_floor(float a)  { return floorf(a); }
__device__ __forceinline__ double t_floor(double a) { return floor(a); }

// Order-preserving key of a finite ratio for the ANCHOR_MIN reduction: larger key = smaller
// ratio, and 0 is never produced for a finite value, so a zero word means "no value".
__device__ __forceinline__ unsigned long long min_key(double r) {
  unsigned long long u = (unsigned long long)__double_as_longlong(r);
  unsigned long long ord = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  return ~ord;
}
__device__ __forceinline__ unsigned long long min_key(float r) { return min_key((double)r); }
__host__ __device__ __forceinline__ double key_to_ratio(unsigned long long key) {
  unsigned long long ord = ~key;
  unsigned long long u = (ord >> 63) ? (ord & 0x7FFFFFFFFFFFFFFFull) : ~ord;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  __builtin_memcpy(&d, &u, 8);
  return d;
#endif
}

// ------------------------------------------------------------------------------------------
// The exact chain: ratio (Eq. 1), binnable test, bin id (§IV.B.1).
// Returns 1 and the bin if binnable, 0 otherwise. |ratio| <= cap also rejects NaN and inf.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int classify_exact(T p, T x, const Consts<T>& c, int& b) {
  // p = +-0 makes the ratio +-inf or NaN, which is never binnable: decided before the divide,
  // whose IEEE special-operand path is slow and diverges the warp
  if (p == (T)0) return 0;
  T d = t_sub(x, p);
  T r = t_div(d, p);
  if (!(t_abs(r) <= c.cap)) return 0;
  T t = t_sub(r, c.a);
  T u = t_mul(t, c.inv_w);
  b = (int)t_floor(u);
  return 1;
}

// Exact error-bound check of §III.C with the multiplier m = 1 + centre (Eq. 4):
// |p*m - x| <= E_T*|x| in T.
template <typename T>
__device__ __forceinline__ bool check_exact(T p, T x, T m, T E_T) {
  T R = t_mul(p, m);
  T e = t_sub(R, x);
  T tol = t_mul(E_T, t_abs(x));
  return t_abs(e) <= tol;
}

// Centre of bin b, a + (b + 1/2) w (§III.B), and the multiplier m = 1 + centre (Eq. 4), in T.
template <typename T>
__device__ __forceinline__ T bin_centre(int b, T a, T w) {
  return t_add(a, t_mul(t_add((T)b, (T)0.5), w));
}
template <typename T>
__device__ __forceinline__ T bin_multiplier(int b, T a, T w) {
  return t_add((T)1, bin_centre<T>(b, a, w));
}

static __device__ __noinline__ int classify_exact_f64_slow(double p, double x, const Consts<double>& c,
                                                   int* b) {
  int bb = 0;
  int k = classify_exact<double>(p, x, c, bb);
  *b = bb;
  return k;
}
static __device__ __noinline__ bool check_exact_f64_slow(double p, double x, double m, double E_T) {
  return check_exact<double>(p, x, m, E_T);
}

// ------------------------------------------------------------------------------------------
// float64 filter-and-refine.
//
// Fast path: p normal with biased exponent ep in [200, 1940] and x finite. With s = 2^(ep-1023):
//   d64 = fl64(x - p)                       (one DSUB; |d64 - d| <= 2^-53 |d|)
//   df  = d64/s truncated to 24 bits         (bit assembly; relative error < 2^-23;
//                                             |d/s| < 2^-126, which includes every subnormal
//                                             d64 since ep >= 200, is taken as 0)
//   pf  = |p|/s = 1.mantissa(p) truncated    (relative error < 2^-23)
//   Df  = fl32(df * rcp.approx(pf)) * sign(p) (rcp.approx: absolute error 2^-23 on [1, 2))
// so |Df - D*| <= 2^-20.8 |D*| + 2^-126 with D* = (x - p)/p exactly. The exact float64 chain
// (two roundings to the ratio, one each to t and u) satisfies
//   |u64 - U| <= 2.01 * 2^-53 (|U| + inv_w |D*|),   U = (D* - a) inv_w,
// and the float32 chain tf = fl(Df - af), uf = fl(tf * inv_wf) satisfies
//   |uf - U| <= 3.01 * 2^-24 |U| + inv_w (2^-20.8 |D*| + 2^-24 |a| + 2^-126).
// Using inv_w |D*| <= (|uf| + inv_w |a|)(1 + 2^-20), everything is bounded by
//   eps = 1.5 * 2^-20 |uf| + (2^-19 inv_w |a| + 2^-60)     (one FMA rounded upward)
// When floor(uf - eps) == floor(uf + eps) (rounded downward / upward), that floor is
// floor(u64), the exact float64 bin. The cap test uses margins 2^-19 the same way.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The float32 ratio estimate Df of the fast path (valid when p has a biased exponent in
// [200, 1940] and x is finite; see above). Returns false when |d/s| >= 2^128.
__device__ __forceinline__ bool ratio_estimate(unsigned ph, unsigned pl, int ep, double p, double x,
                                               float& Df) {
  const double d = __dsub_rn(x, p);
  const unsigned dh = (unsigned)__double2hiint(d), dl = (unsigned)__double2loint(d);
  const int e32 = (int)((dh >> 20) & 0x7FFu) - ep + 127;
  const unsigned dmant = __funnelshift_r(dl, dh, 29) & 0x7FFFFFu;
  const unsigned dsign = dh & 0x80000000u;
  const float df = __uint_as_float(e32 > 0 ? (dsign | ((unsigned)e32 << 23) | dmant) : dsign);
  const float pf = __uint_as_float(0x3F800000u | (__funnelshift_r(pl, ph, 29) & 0x7FFFFFu));
  Df = __uint_as_float(__float_as_uint(__fmul_rn(df, rcp_approx(pf))) ^ (ph & 0x80000000u));
  return e32 < 255;
}

// Bin of (p, x) for float64: 1 and the bin if binnable, else 0. Equal to classify_exact<double>.
__device__ __forceinline__ int classify_f64(double p, double x, const Consts<double>& c, int& b) {
  const unsigned ph = (unsigned)__double2hiint(p), pl = (unsigned)__double2loint(p);
  const unsigned xh = (unsigned)__double2hiint(x);
  const int ep = (int)((ph >> 20) & 0x7FFu);
  const int ex = (int)((xh >> 20) & 0x7FFu);
  if ((unsigned)(ep - 200) <= 1740u && ex != 0x7FF) {
    float Df;
    if (!ratio_estimate(ph, pl, ep, p, x, Df)) return 0;   // |d/s| >= 2^128: far beyond the cap
    const float aD = fabsf(Df);
    if (aD > c.cap_hi) return 0;                           // certainly |ratio| > cap
    if (aD <= c.cap_lo) {                                  // certainly binnable
      const float uf = __fmul_rn(__fsub_rn(Df, c.af), c.inv_wf);
      const float eps = __fmaf_ru(0x1.8p-20f, fabsf(uf), c.K0);
      const float lo = floorf(__fsub_rd(uf, eps));
      const float hi = floorf(__fadd_ru(uf, eps));
      if (lo == hi && lo < 4194304.0f) {
        b = __float_as_int(__fadd_rn(lo, 12582912.0f)) - 0x4B400000;   // exact for |lo| < 2^22
        return 1;
      }
    }
  } else if ((ph << 1) == 0u && pl == 0u) {
    return 0;                                              // p = +-0: ratio is +-inf or NaN
  } else if (ep == 0x7FF || ex == 0x7FF) {
    return 0;                                              // non-finite input
  }
  return classify_exact_f64_slow(p, x, c, &b);
}

// Error-bound check of §III.C for float64 points in a selected bin, decided in ratio space.
// Dividing the exact check |fl(fl(p*m) - x)| <= fl(E_T*|x|) by |p| gives, with
// G* = c' - D* (c' = m - 1 exactly, D* = (x - p)/p) and H* = E_T |1 + D*|:
//   ok  <=>  |G* + eta| <= H* (1 + theta),  |eta| <= 2^-52 (|m| + |G*|),  |theta| <= 2^-53.
// The float32 estimates G = fl(cf - Df), cf = fl32(fl64(m - 1)), and
// H = fl(Ef * |fl(1 + Df)|) satisfy
//   |G - G*| <= 2^-23.9 |cf| + 2^-20.7 |Df| + 2^-24 |G| + 2^-125,
//   |H - H*| <= 3 * 2^-24 H + 2^-20.7 E_T |Df|.
// delta = 2^-23 (|cf| + |G|) + 2^-20 |Df| + 2^-50 |cf| + 2^-49 covers the first line and eta;
// deltaH = 2^-21 H + 2^-20 Ef |Df| + 2^-100 covers the second. If |G| + delta < H - deltaH the
// exact check passes; if |G| - delta > H + deltaH it fails; otherwise the exact float64 check
// decides. (All bound arithmetic rounds away from the decision.)
// The check with that rule, falling back to the exact float64 sequence when it cannot decide.
__device__ __forceinline__ bool check_f64(double p, double x, double m, float cf,
                                          const Consts<double>& c) {
  const unsigned ph = (unsigned)__double2hiint(p), pl = (unsigned)__double2loint(p);
  const unsigned xh = (unsigned)__double2hiint(x);
  const int ep = (int)((ph >> 20) & 0x7FFu);
  const int ex = (int)((xh >> 20) & 0x7FFu);
  if ((unsigned)(ep - 200) <= 1740u && (unsigned)(ex - 100) <= 1840u) {
    float Df;
    if (ratio_estimate(ph, pl, ep, p, x, Df)) {
      const float aDf = fabsf(Df);
      const float G = __fsub_rn(cf, Df);
      const float aG = fabsf(G);
      const float H = __fmul_rn(c.Ef, fabsf(__fadd_rn(1.0f, Df)));
      const float delta = __fmaf_ru(0x1p-23f, __fadd_ru(fabsf(cf), aG),
                                    __fmaf_ru(0x1p-20f, aDf,
                                              __fmaf_ru(0x1p-50f, fabsf(cf), 0x1p-49f)));
      const float dH = __fmaf_ru(0x1p-21f, H, __fmaf_ru(0x1p-20f * c.Ef, aDf, 0x1p-100f));
      if (__fadd_ru(aG, delta) < __fsub_rd(H, dH)) return true;
      if (__fsub_rd(aG, delta) > __fadd_ru(H, dH)) return false;
    }
  }
  return check_exact_f64_slow(p, x, m, c.E_T);
}

// K1's fused float64 step: the bin of (p, x) as classify_f64's estimate decides it and, for a bin in
// the code window, the check of §III.C against that bin's own centre, decided from the same
// ratio estimate Df. The multiplier is estimated in float32 from the bin id:
//   v = b + 1/2 (exact), Q = fl32(v * wf), cfe = fl32(af + Q),
// while the exact sequence uses c' = m - 1, m = fl64(1 + fl64(a + fl64(v * w))). Then
//   |c' - (a + v w)|  <= 2^-51 (1 + |a| + 2 |v w|)                       (three roundings),
//   |cfe - (a + v w)| <= 1.07 * 2^-24 |cfe| + 2^-24 |a| + 2.0001 * 2^-24 |v w|,
// and as |a| <= |af| (1 + 2^-23), |v w| <= |Q| (1 + 2^-22):
//   |cfe - c'| <= Kc = 2^-22 (|cfe| + |af| + 2 |Q|) + 2^-50               (rounded upward),
// which takes the place of the rounding of cf in check_f64's bound: the same decision rule
// with G = fl(cfe - Df) and delta + Kc is exact. The terms of delta + Kc and dH are regrouped
// below into one per-bin term and one term in |Df| (each rounded upward, so every comparison
// implies the one it replaces).
// Returns 1 (binnable: the bin, and pass when the bin is in the window, decided), 0 (with
// ZERO_P: p = +-0, whose ratio is +-inf or NaN and never binnable) or 2 (the exact sequences must
// decide the point; p = +-0 too without ZERO_P).
template <bool ZERO_P = true>
__device__ __forceinline__ int classify_check_f64_fast(double p, double x, const Consts<double>& c,
                                                       int cbase, int& b, bool& pass) {
  // computed without branches: every quantity below is harmless for any input bits, and the
  // outcome is selected at the end
  const unsigned ph = (unsigned)__double2hiint(p), pl = (unsigned)__double2loint(p);
  const unsigned xh = (unsigned)__double2hiint(x);
  const int ep = (int)((ph >> 20) & 0x7FFu);
  const int ex = (int)((xh >> 20) & 0x7FFu);
  float Df;
  const bool est = ratio_estimate(ph, pl, ep, p, x, Df);   // false: |d/s| >= 2^128
  const float aD = fabsf(Df);
  const float uf = __fmul_rn(__fsub_rn(Df, c.af), c.inv_wf);
  const float eps = __fmaf_ru(0x1.8p-20f, fabsf(uf), c.K0);
  const float lo = floorf(__fsub_rd(uf, eps));
  const float hi = floorf(__fadd_ru(uf, eps));
  b = __float_as_int(__fadd_rn(lo, 12582912.0f)) - 0x4B400000;     // exact for |lo| < 2^22
  const float Q = __fmul_rn(__fadd_rn(lo, 0.5f), c.wf);             // lo + 1/2 exact
  const float cfe = __fadd_rn(c.af, Q);
  // Pb >= 2^-23 |cfe| + 2^-50 |cfe| + 2^-49 + Kc + 2^-100: the parts of delta and dH that depend
  // on the bin alone; T1 adds the parts proportional to |Df| (2^-20 (1 + Ef) |Df|)
  const float Pb = __fmaf_ru(fabsf(cfe), c.kA, __fmaf_ru(fabsf(Q), 0x1p-21f, c.C0));
  const float T1 = __fmaf_ru(aD, c.k1, Pb);
  const float aG = fabsf(__fsub_rn(cfe, Df));
  const float H = __fmul_rn(c.Ef, fabsf(__fadd_rn(1.0f, Df)));
  // |G| + delta < H - dH, i.e. |G| (1 + 2^-23) + T1 < H (1 - 2^-21): the check passes;
  // |G| - delta > H + dH, i.e. |G| (1 - 2^-23) > H (1 + 2^-21) + T1: it fails
  const bool yes = __fmaf_ru(aG, 0x1.000002p+0f, T1) < __fmul_rd(H, 0x1.fffffp-1f);
  const bool no = __fmul_rd(aG, 0x1.fffffcp-1f) > __fmaf_ru(H, 0x1.000008p+0f, T1);
  pass = yes;
  // estimate valid (a non-finite x gives |Df| >= 2^106 or est false: beyond cap_lo, which is at
  // most 2^100 and, with E < 1, below 2^22)
  const bool in_range = (unsigned)(ep - 200) <= 1740u;
  // binnable with its bin decided: the estimate is valid and finite, certainly within the cap,
  // and both ends of its error interval fall in one bin
  const bool sure = in_range && est && aD <= c.cap_lo && lo == hi && lo < 4194304.0f;
  const bool outside = (unsigned)(b - cbase) >= (unsigned)CODE_BINS;     // no check needed
  const bool decided = (unsigned)(ex - 100) <= 1840u && (yes || no);     // check decided
  // everything else (inputs outside the estimate's range, ratios near or beyond the cap, bins
  // or checks the estimate cannot decide) is rare and goes to the exact sequences, which the
  // callers settle 32 at a time
  if constexpr (ZERO_P) {
    const bool pzero = ((ph << 1) | pl) == 0u;                         // ratio +-inf or NaN
    return (sure && (outside || decided)) ? 1 : (pzero ? 0 : 2);
  } else {
    return (sure && (outside || decided)) ? 1 : 2;
  }
}

// ------------------------------------------------------------------------------------------
// Block-wide helpers
// ------------------------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V warp_incl_scan(V v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    V t = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += t;
  }
  return v;
}

}  // namespace nmk
