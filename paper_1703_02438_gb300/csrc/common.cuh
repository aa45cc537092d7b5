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
constexpr int RW_BINS = 8192;                   // K3 shared-memory rank window
constexpr int MT_SMEM = 1024;                   // K3 multipliers kept in shared memory
constexpr int DM_SMEM = 4096;                   // K4 multipliers kept in shared memory
constexpr int TILE_THREADS = 512;               // K3/K4 block size
constexpr int EPT = SUB / TILE_THREADS;         // elements per thread per tile (8)
constexpr int NCHUNK = EPT * (TILE_THREADS / 32); // 32-element chunks per tile (128)
constexpr unsigned KEY_BIAS = 0x40000000u;      // bin-range keys: 0 means "no value"

// Workspace control block (first 256 bytes of the workspace). Zero at entry of every
// compression; the kernels restore the zero state of every field they accumulate into.
struct Ctrl {
  unsigned int bmin_key;        // max over binnable points of (KEY_BIAS - bin)
  unsigned int bmax_key;        // max over binnable points of (bin + KEY_BIAS)
  unsigned long long amin_key;  // ANCHOR_MIN: max of ~orderable(ratio)
  unsigned int ticket;          // K3 dynamic tile counter (reset by K1)
  int error;                    // device-side NUMARCK_ERR_* of the current call
  // written by K2 for K3 (plain stores; no reset needed)
  int any;                      // 1 if at least one point is binnable
  int sel_bmin, sel_bmax;       // bin range of the binnable points
  int n_sel;                    // selected bins
  int pad0;
  double a;                     // grid anchor (the T value, widened)
  unsigned int win_err;         // a bin fell outside the histogram window (never expected)
  unsigned int pad1[49];
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
  // float64 estimate: af = fl32(a), inv_wf = fl32(inv_w), Ef = fl32(E_T),
  // cap_lo <= cap (1 - 2^-19), cap_hi >= cap (1 + 2^-19), K1 >= 2^-20 inv_w,
  // K0 >= 2^-23 inv_w |a| + 2^-100 (all rounded away from the decision)
  float af, inv_wf, Ef, cap_lo, cap_hi, K1, K0;
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
// Fast path applies when p and x are normal with biased exponents in [100, 1940] and differ
// by at most 9 (|x/p| in (2^-10, 2^10)); everything else takes the exact float64 path.
// Let s = 2^(ep-1023). Then
//   d/s  = (x - p)/s is computed EXACTLY as a 64-bit integer (aligned mantissas, < 2^62) and
//          truncated to 24 bits:            df = (d/s)(1 - tau),  0 <= tau < 2^-23
//   |p|/s = 1.mantissa(p) truncated:         pf = (|p|/s)(1 - tau'), 0 <= tau' < 2^-23
//   Df = __fdividef(df, pf) * sign(p):  |Df - D*| <= 2^-21 |D*|   (2-ulp divide), D* = d/p real
// The exact float64 chain (two roundings to the ratio, one each to t and u) satisfies
//   |u64 - U| <= 2.01 * 2^-53 (|U| + inv_w |D*|),   U = (D* - a) inv_w (real),
// and the float32 chain tf = fl(Df - af), uf = fl(tf * inv_wf) satisfies
//   |uf - U| <= 3.01 * 2^-24 |U| + inv_w (2^-21 |D*| + 2^-24 |a|) (1 + 2^-22).
// Hence |uf - u64| <= eps = 2^-20 inv_w |Df| + 2^-22 |uf| + 2^-23 inv_w |a| (+ 2^-100),
// evaluated with upward rounding (each term carries a factor >= 2 of slack). When
// floor(uf - eps) == floor(uf + eps) (downward / upward rounded), that floor IS floor(u64).
// The cap test is decided the same way with the 2^-19 margins in cap_lo / cap_hi.
// ------------------------------------------------------------------------------------------
struct Est {
  float df;     // (x - p)/s, signed
  float pf;     // |p|/s in [1, 2)
  float xf;     // |x|/s
  int psign;    // sign bit of p
  int fast;     // 1 if the estimate decided the bin (df/pf/xf valid)
};

__device__ __forceinline__ int classify_f64(double p, double x, const Consts<double>& c, int& b,
                                            Est& est) {
  est.fast = 0;
  const unsigned long long pb = (unsigned long long)__double_as_longlong(p);
  const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
  const int ep = (int)((pb >> 52) & 0x7FF);
  const int ex = (int)((xb >> 52) & 0x7FF);
  // p = +-0: ratio is +-inf or NaN; any non-finite input: ratio is inf or NaN.
  if ((pb << 1) == 0 || ep == 0x7FF || ex == 0x7FF) return 0;
  const int de = ex - ep;
  if (ep >= 100 && ex >= 100 && ep <= 1940 && ex <= 1940 && de >= -9 && de <= 9) {
    const unsigned long long MANT = 0x000FFFFFFFFFFFFFull, HID = 0x0010000000000000ull;
    const int sx = de > 0 ? de : 0;
    const int sp = de < 0 ? -de : 0;
    long long X = (long long)(((xb & MANT) | HID) << sx);
    long long P = (long long)(((pb & MANT) | HID) << sp);
    if (xb >> 63) X = -X;
    if (pb >> 63) P = -P;
    const long long Di = X - P;  // d = Di * 2^(min(ex,ep) - 1075), exactly
    float df = 0.0f;
    if (Di != 0) {
      const unsigned long long mag = Di < 0 ? (unsigned long long)(-Di) : (unsigned long long)Di;
      const int lz = __clzll((long long)mag);
      const unsigned m24 = (unsigned)((mag << lz) >> 40);
      const unsigned bexp = (unsigned)((63 - lz) - sp + 75);   // in [66, 137]
      df = __uint_as_float((bexp << 23) | (m24 & 0x7FFFFFu) | (Di < 0 ? 0x80000000u : 0u));
    }
    const float pf = __uint_as_float(0x3F800000u | (unsigned)((pb >> 29) & 0x7FFFFFu));
    float Df = __fdividef(df, pf);
    if (pb >> 63) Df = -Df;
    const float aD = fabsf(Df);
    if (aD > c.cap_hi) return 0;                 // certainly |ratio| > cap
    if (aD <= c.cap_lo) {                        // certainly binnable
      const float tf = __fsub_rn(Df, c.af);
      const float uf = __fmul_rn(tf, c.inv_wf);
      const float eps = __fadd_ru(__fadd_ru(__fmul_ru(c.K1, aD), __fmul_ru(0x1p-22f, fabsf(uf))),
                                  c.K0);
      const float lo = floorf(__fsub_rd(uf, eps));
      const float hi = floorf(__fadd_ru(uf, eps));
      if (lo == hi) {
        b = (int)lo;
        est.fast = 1;
        est.df = df;
        est.pf = pf;
        est.psign = (int)(pb >> 63);
        est.xf = __uint_as_float(((unsigned)(de + 127) << 23) | (unsigned)((xb >> 29) & 0x7FFFFFu));
        return 1;
      }
    }
  }
  return classify_exact_f64_slow(p, x, c, &b);
}

// Error-bound check for float64 with the estimate of classify_f64.
// With e* = p*m - x = p*c' - d (c' = m - 1 exactly, real), in units of s:
//   pc = fl32(sign(p) pf * cf), cf = fl32(fl64(m - 1)):  |pc - p c'/s| <= 2^-22 |pc| (1+2^-21)
//   ef = fl32(pc - df):   |ef - e*/s| <= 2^-21|pc| + 2^-22|df| + 2^-23|ef| =: beta
//   float64: |e64 - e*|/s <= 2^-50 (pf (1 + |cf|) + |ef|) (one rounding in p*m, one in R - x)
//   tolf = fl32(Ef * xf):  tol64/s in [tolf (1 - 2^-21), tolf (1 + 2^-21)]
// so |ef| + beta' < tolf (1 - 2^-21) proves |e64| <= tol64, and |ef| - beta' > tolf (1 + 2^-21)
// proves the opposite; otherwise the exact float64 check decides.
__device__ __forceinline__ bool check_f64(double p, double x, double m, float cf,
                                          const Consts<double>& c, const Est& est) {
  if (est.fast) {
    const float ps = est.psign ? -est.pf : est.pf;
    const float pc = __fmul_rn(ps, cf);
    const float ef = __fsub_rn(pc, est.df);
    const float tolf = __fmul_rn(c.Ef, est.xf);
    const float aef = fabsf(ef);
    const float beta = __fadd_ru(
        __fadd_ru(__fmul_ru(0x1p-21f, fabsf(pc)), __fmul_ru(0x1p-22f, fabsf(est.df))),
        __fadd_ru(__fmul_ru(0x1p-23f, aef),
                  __fmul_ru(0x1p-50f, __fadd_ru(__fmul_ru(est.pf, __fadd_ru(1.0f, fabsf(cf))),
                                                aef))));
    if (__fadd_ru(aef, beta) < __fmul_rd(tolf, 1.0f - 0x1p-21f)) return true;
    if (__fsub_rd(aef, beta) > __fmul_ru(tolf, 1.0f + 0x1p-21f)) return false;
  }
  return check_exact_f64_slow(p, x, m, c.E_T);
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
