/* numarck_cpu.c — a multi-threaded CPU implementation of NUMARCK compression and decompression,
 * used as the all-cores CPU baseline of the benchmark and as a second CPU check of the oracle.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY. It is written in plain C from the same readings of the
 * paper as the numpy oracle (oracle/numarck_oracle.py), shares no code with the GPU library, and
 * produces the same blob bytes as the oracle (tests/test_cpu_baseline.py checks that). Only the
 * test suite and bench.py's cpu_baseline leg load it.
 *
 * Source: Z. Yuan et al., "Parallel Implementation of Lossy Data Compression for Temporal Data
 * Sets", arXiv 1703.02438. Steps: change ratio (Eq. 1, §III.A), bins of width 2E and the
 * histogram (§IV.B.1), top-k selection (§IV.B.1), indexing with the element-wise error-bound
 * check (§III.C, Eq. 4 read as R = prev (1 + centre)), byte-aligned index blocks of B-bit indices
 * (§IV.C) and the incompressible table with its offsets (§III.C, §IV.C); the automatic index
 * length of §IV.B.2 (Eqs. 5, 6); decompression (§III.E).
 *
 * Parallel structure (the paper's MPI decomposition, §IV, on threads of one host): contiguous
 * chunks of the elements per thread for the ratio/bin pass with per-thread histograms merged
 * afterwards (the paper's MPI_Allreduce), top-k on one thread (replicated in the paper), then
 * 4096-element tiles of the index blocks in parallel for indexing and packing, a prefix over the
 * tiles' incompressible counts, and the copy of the incompressible values per tile.
 *
 * Arithmetic: every floating-point operation is one C operation in the element type (float or
 * double), compiled with -ffp-contract=off (no fused multiply-add) and without fast-math, so it
 * is rounded once, to nearest even, in the order written.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NC_MAGIC 0x314B4D4Eu
#define NC_VERSION 1u
#define NC_HEADER 256
#define NC_ALIGN 256
#define NC_SUB 4096
#define NC_WIN_LOG2 21
#define NC_MARGIN 8
#define NC_HBINS ((1 << (NC_WIN_LOG2 + 1)) + 2 * NC_MARGIN + 8)

enum { NC_OK = 0, NC_EINVAL = 1, NC_ECAP = 2, NC_ENOMEM = 7, NC_ECORRUPT = 4 };

static int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* ---------------------------------------------------------------------------------------- */
/* Blob layout (§IV.C block layout, §IV.D / Fig. 2 arrays, plus the header and the sub-block
 * table of this format).                                                                    */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
  int64_t n, L, B, epb, nblocks, nsub, block_stride, index_bytes, last;
  int64_t off_centres, off_idx_off, off_inc_off, off_sub_off, off_index, off_exact;
} layout_t;

static layout_t make_layout(int64_t n, int L, int B, int64_t block_bytes) {
  layout_t g;
  memset(&g, 0, sizeof(g));
  g.n = n;
  g.L = L;
  g.B = B;
  g.epb = 8 * block_bytes / B;
  g.nblocks = n > 0 ? cdiv(n, g.epb) : 0;
  g.last = g.nblocks ? n - (g.nblocks - 1) * g.epb : 0;
  g.nsub = g.nblocks ? (g.nblocks - 1) * cdiv(g.epb, NC_SUB) + cdiv(g.last, NC_SUB) : 0;
  g.block_stride = rup(cdiv(g.epb * B, 8), 16);
  g.index_bytes = g.nblocks ? (g.nblocks - 1) * g.block_stride + rup(cdiv(g.last * B, 8), 16) : 0;
  g.off_centres = NC_HEADER;
  g.off_idx_off = rup(g.off_centres + ((int64_t)1 << B) * L, NC_ALIGN);
  g.off_inc_off = rup(g.off_idx_off + (g.nblocks + 1) * 8, NC_ALIGN);
  g.off_sub_off = rup(g.off_inc_off + (g.nblocks + 1) * 8, NC_ALIGN);
  g.off_index = rup(g.off_sub_off + g.nsub * 8, NC_ALIGN);
  g.off_exact = rup(g.off_index + g.index_bytes, NC_ALIGN);
  return g;
}

size_t ncpu_compress_bound(int64_t n, int dtype, int B, int64_t block_bytes) {
  const int L = dtype ? 8 : 4;
  if (n < 0 || B < 0 || B > 16 || block_bytes < 2) return 0;
  int64_t off = 0;
  for (int b = B ? B : 1; b <= (B ? B : 16); ++b) {
    const layout_t g = make_layout(n, L, b, block_bytes);
    if (g.off_exact > off) off = g.off_exact;
  }
  return (size_t)(off + n * L);
}

/* ---------------------------------------------------------------------------------------- */
/* A minimal parallel-for over [0, count) on `threads` POSIX threads (static chunks).        */
/* ---------------------------------------------------------------------------------------- */
typedef void (*body_fn)(void* ctx, int64_t lo, int64_t hi, int tid);
typedef struct {
  body_fn fn;
  void* ctx;
  int64_t lo, hi;
  int tid;
} task_t;

static void* run_task(void* p) {
  task_t* t = (task_t*)p;
  if (t->lo < t->hi) t->fn(t->ctx, t->lo, t->hi, t->tid);
  return NULL;
}

static int parallel_for(int threads, int64_t count, body_fn fn, void* ctx) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  task_t tasks[256];
  pthread_t th[256];
  int started[256];
  for (int i = 0; i < threads; ++i) {
    tasks[i].fn = fn;
    tasks[i].ctx = ctx;
    tasks[i].lo = count * i / threads;
    tasks[i].hi = count * (i + 1) / threads;
    tasks[i].tid = i;
    started[i] = 0;
  }
  for (int i = 1; i < threads; ++i)
    started[i] = pthread_create(&th[i], NULL, run_task, &tasks[i]) == 0;
  run_task(&tasks[0]);
  for (int i = 1; i < threads; ++i) {
    if (started[i])
      pthread_join(th[i], NULL);
    else
      run_task(&tasks[i]);             /* a thread that could not start: run its part here */
  }
  return NC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* The element-type-specific steps, written once for float and once for double.              */
/* ---------------------------------------------------------------------------------------- */
#define NC_DEFINE(T, SUFFIX, FLOOR, FABS, ISFINITE)                                            \
  typedef struct {                                                                             \
    const T* prev;                                                                             \
    const T* cur;                                                                              \
    T E_T, w, inv_w, cap, a;                                                                   \
    int32_t* bins;          /* bin id per element; INT32_MIN: not binnable */                  \
    uint32_t* hist;         /* per-thread dense windows of NC_HBINS counts */                  \
    int64_t hbase;          /* bin of window entry 0 */                                        \
    int64_t* tmin;          /* per-thread smallest / largest bin seen */                       \
    int64_t* tmax;                                                                             \
    T* minr;                /* per-thread smallest binnable ratio (MIN grid) */                \
    int* anyr;                                                                                 \
    int err;                                                                                   \
  } pass1_##SUFFIX;                                                                            \
                                                                                               \
  /* Eq. 1 ratio and the binnable test, in T */                                                \
  static int ratio_##SUFFIX(T p, T x, T cap, T* r) {                                           \
    const T d = x - p;                                                                         \
    const T q = d / p;                                                                         \
    *r = q;                                                                                    \
    return ISFINITE(q) && FABS(q) <= cap;                                                      \
  }                                                                                            \
                                                                                               \
  static void min_body_##SUFFIX(void* vctx, int64_t lo, int64_t hi, int tid) {                 \
    pass1_##SUFFIX* c = (pass1_##SUFFIX*)vctx;                                                 \
    T best = 0;                                                                                \
    int any = 0;                                                                               \
    for (int64_t j = lo; j < hi; ++j) {                                                        \
      T r;                                                                                     \
      if (ratio_##SUFFIX(c->prev[j], c->cur[j], c->cap, &r) && (!any || r < best)) {           \
        best = r;                                                                              \
        any = 1;                                                                               \
      }                                                                                        \
    }                                                                                          \
    c->minr[tid] = best;                                                                       \
    c->anyr[tid] = any;                                                                        \
  }                                                                                            \
                                                                                               \
  /* bin = floor((ratio - a) * (1 / 2E)) (§IV.B.1) and the per-thread histogram */             \
  static void bin_body_##SUFFIX(void* vctx, int64_t lo, int64_t hi, int tid) {                 \
    pass1_##SUFFIX* c = (pass1_##SUFFIX*)vctx;                                                 \
    uint32_t* h = c->hist + (size_t)tid * NC_HBINS;                                            \
    int64_t mn = INT64_MAX, mx = INT64_MIN;                                                    \
    for (int64_t j = lo; j < hi; ++j) {                                                        \
      T r;                                                                                     \
      if (!ratio_##SUFFIX(c->prev[j], c->cur[j], c->cap, &r)) {                                \
        c->bins[j] = INT32_MIN;                                                                \
        continue;                                                                              \
      }                                                                                        \
      const T t = r - c->a;                                                                    \
      const T u = t * c->inv_w;                                                                \
      const int64_t b = (int64_t)FLOOR(u);                                                     \
      const int64_t k = b - c->hbase;                                                          \
      if (k < 0 || k >= NC_HBINS) { c->err = 1; c->bins[j] = INT32_MIN; continue; }            \
      c->bins[j] = (int32_t)b;                                                                 \
      h[k] += 1u;                                                                              \
      if (b < mn) mn = b;                                                                      \
      if (b > mx) mx = b;                                                                      \
    }                                                                                          \
    c->tmin[tid] = mn;                                                                         \
    c->tmax[tid] = mx;                                                                         \
  }                                                                                            \
                                                                                               \
  typedef struct {                                                                             \
    const T* prev;                                                                             \
    const T* cur;                                                                              \
    const int32_t* bins;                                                                       \
    const int32_t* rank;      /* rank of bin (b - rbase), -1 if not selected */                \
    int64_t rbase, rlen;                                                                       \
    const T* mult;            /* m_r = 1 + centre_r */                                         \
    T E_T;                                                                                     \
    layout_t g;                                                                                \
    unsigned char* blob;                                                                       \
    uint8_t* marker;          /* 1 per incompressible element */                               \
    int64_t* tile_count;                                                                       \
  } pass2_##SUFFIX;                                                                            \
                                                                                               \
  /* §III.C indexing with the check |prev m - cur| <= E |cur| in T, and §IV.C bit packing, one  \
   * 4096-element tile of an index block at a time (tiles start on byte boundaries) */          \
  static void assign_body_##SUFFIX(void* vctx, int64_t lo, int64_t hi, int tid) {              \
    (void)tid;                                                                                 \
    pass2_##SUFFIX* c = (pass2_##SUFFIX*)vctx;                                                 \
    const layout_t* g = &c->g;                                                                 \
    const int64_t spb = cdiv(g->epb, NC_SUB);                                                  \
    const uint32_t M = (1u << g->B) - 1u;                                                      \
    for (int64_t gt = lo; gt < hi; ++gt) {                                                     \
      const int64_t q = gt / spb, t = gt - q * spb;                                            \
      const int64_t j0 = q * g->epb + t * NC_SUB;                                              \
      int64_t j1 = j0 + NC_SUB;                                                                \
      const int64_t bend = (q + 1) * g->epb < g->n ? (q + 1) * g->epb : g->n;                  \
      if (j1 > bend) j1 = bend;                                                                \
      unsigned char* img = c->blob + g->off_index + q * g->block_stride + t * (NC_SUB / 8) * g->B; \
      uint64_t acc = 0;                                                                        \
      int nacc = 0;                                                                            \
      int64_t cnt = 0;                                                                         \
      for (int64_t j = j0; j < j1; ++j) {                                                      \
        uint32_t idx = M;                                                                      \
        const int32_t b = c->bins[j];                                                          \
        if (b != INT32_MIN) {                                                                  \
          const int64_t k = (int64_t)b - c->rbase;                                             \
          if (k >= 0 && k < c->rlen && c->rank[k] >= 0) {                                      \
            const int32_t r = c->rank[k];                                                      \
            const T R = c->prev[j] * c->mult[r];                                               \
            const T e = R - c->cur[j];                                                         \
            const T tol = c->E_T * FABS(c->cur[j]);                                            \
            if (FABS(e) <= tol) idx = (uint32_t)r;                                             \
          }                                                                                    \
        }                                                                                      \
        c->marker[j] = idx == M;                                                               \
        cnt += idx == M;                                                                       \
        acc |= (uint64_t)idx << nacc;                                                          \
        nacc += (int)g->B;                                                                     \
        while (nacc >= 8) {                                                                    \
          *img++ = (unsigned char)(acc & 0xFFu);                                               \
          acc >>= 8;                                                                           \
          nacc -= 8;                                                                           \
        }                                                                                      \
      }                                                                                        \
      if (nacc > 0) *img = (unsigned char)(acc & 0xFFu);                                       \
      c->tile_count[gt] = cnt;                                                                 \
    }                                                                                          \
  }                                                                                            \
                                                                                               \
  typedef struct {                                                                             \
    const T* cur;                                                                              \
    const uint8_t* marker;                                                                     \
    const int64_t* tile_off; /* incompressible values before each tile */                      \
    layout_t g;                                                                                \
    T* exact;                                                                                  \
  } pass3_##SUFFIX;                                                                            \
                                                                                               \
  static void exact_body_##SUFFIX(void* vctx, int64_t lo, int64_t hi, int tid) {               \
    (void)tid;                                                                                 \
    pass3_##SUFFIX* c = (pass3_##SUFFIX*)vctx;                                                 \
    const layout_t* g = &c->g;                                                                 \
    const int64_t spb = cdiv(g->epb, NC_SUB);                                                  \
    for (int64_t gt = lo; gt < hi; ++gt) {                                                     \
      const int64_t q = gt / spb, t = gt - q * spb;                                            \
      const int64_t j0 = q * g->epb + t * NC_SUB;                                              \
      int64_t j1 = j0 + NC_SUB;                                                                \
      const int64_t bend = (q + 1) * g->epb < g->n ? (q + 1) * g->epb : g->n;                  \
      if (j1 > bend) j1 = bend;                                                                \
      int64_t o = c->tile_off[gt];                                                             \
      for (int64_t j = j0; j < j1; ++j)                                                        \
        if (c->marker[j]) memcpy(&c->exact[o++], &c->cur[j], sizeof(T));                       \
    }                                                                                          \
  }                                                                                            \
                                                                                               \
  typedef struct {                                                                             \
    const T* prev;                                                                             \
    T* out;                                                                                    \
    const unsigned char* blob;                                                                 \
    layout_t g;                                                                                \
    const int64_t* sub_off;                                                                    \
    const T* mult;                                                                             \
    const T* exact;                                                                            \
    int64_t n_inc;                                                                             \
    int err;                                                                                   \
  } pass4_##SUFFIX;                                                                            \
                                                                                               \
  /* §III.E: R = prev * (1 + centre[idx]), or the next incompressible value */                 \
  static void decode_body_##SUFFIX(void* vctx, int64_t lo, int64_t hi, int tid) {              \
    (void)tid;                                                                                 \
    pass4_##SUFFIX* c = (pass4_##SUFFIX*)vctx;                                                 \
    const layout_t* g = &c->g;                                                                 \
    const int64_t spb = cdiv(g->epb, NC_SUB);                                                  \
    const uint32_t M = (1u << g->B) - 1u;                                                      \
    for (int64_t gt = lo; gt < hi; ++gt) {                                                     \
      const int64_t q = gt / spb, t = gt - q * spb;                                            \
      const int64_t j0 = q * g->epb + t * NC_SUB;                                              \
      int64_t j1 = j0 + NC_SUB;                                                                \
      const int64_t bend = (q + 1) * g->epb < g->n ? (q + 1) * g->epb : g->n;                  \
      if (j1 > bend) j1 = bend;                                                                \
      const unsigned char* img =                                                               \
          c->blob + g->off_index + q * g->block_stride + t * (NC_SUB / 8) * g->B;              \
      int64_t o = c->sub_off[gt];                                                              \
      uint64_t acc = 0;                                                                        \
      int nacc = 0;                                                                            \
      for (int64_t j = j0; j < j1; ++j) {                                                      \
        while (nacc < (int)g->B) {                                                             \
          acc |= (uint64_t)(*img++) << nacc;                                                   \
          nacc += 8;                                                                           \
        }                                                                                      \
        const uint32_t idx = (uint32_t)(acc & M);                                              \
        acc >>= g->B;                                                                          \
        nacc -= (int)g->B;                                                                     \
        if (idx == M) {                                                                        \
          if (o < 0 || o >= c->n_inc) { c->err = 1; return; }                                  \
          memcpy(&c->out[j], &c->exact[o++], sizeof(T));                                       \
        } else {                                                                               \
          c->out[j] = c->prev[j] * c->mult[idx];                                               \
        }                                                                                      \
      }                                                                                        \
    }                                                                                          \
  }

NC_DEFINE(float, f32, floorf, fabsf, isfinite)
NC_DEFINE(double, f64, floor, fabs, isfinite)

/* ---------------------------------------------------------------------------------------- */
/* Header (the documented 256-byte header: little-endian fields, then zero bytes).           */
/* ---------------------------------------------------------------------------------------- */
static void put32(unsigned char* p, uint32_t v) { memcpy(p, &v, 4); }
static void put64(unsigned char* p, int64_t v) { memcpy(p, &v, 8); }
static void putd(unsigned char* p, double v) { memcpy(p, &v, 8); }

static void write_header(unsigned char* h, const layout_t* g, int dtype, double E, int anchor,
                         int64_t block_bytes, int64_t n_sel, int64_t n_inc, double a) {
  memset(h, 0, NC_HEADER);
  put32(h + 0, NC_MAGIC);
  put32(h + 4, NC_VERSION);
  put32(h + 8, (uint32_t)dtype);
  put32(h + 12, (uint32_t)g->B);
  putd(h + 16, E);
  put32(h + 24, (uint32_t)anchor);
  put32(h + 28, 0u);
  put64(h + 32, g->n);
  put64(h + 40, block_bytes);
  put64(h + 48, g->epb);
  put64(h + 56, g->nblocks);
  put64(h + 64, NC_SUB);
  put64(h + 72, g->nsub);
  put64(h + 80, n_sel);
  put64(h + 88, n_inc);
  putd(h + 96, a);
  put64(h + 104, g->block_stride);
  put64(h + 112, g->off_centres);
  put64(h + 120, g->off_idx_off);
  put64(h + 128, g->off_inc_off);
  put64(h + 136, g->off_sub_off);
  put64(h + 144, g->off_index);
  put64(h + 152, g->off_exact);
  put64(h + 160, g->off_exact + n_inc * g->L);
}

/* top-k order: count descending, then bin ascending (reading R5b) */
typedef struct { int64_t bin, count; } bc_t;
static int by_count_then_bin(const void* x, const void* y) {
  const bc_t* a = (const bc_t*)x;
  const bc_t* b = (const bc_t*)y;
  if (a->count != b->count) return a->count > b->count ? -1 : 1;
  return a->bin < b->bin ? -1 : (a->bin > b->bin);
}
static int by_bin(const void* x, const void* y) {
  const int64_t a = ((const bc_t*)x)->bin, b = ((const bc_t*)y)->bin;
  return a < b ? -1 : (a > b);
}
static int by_count_desc(const void* x, const void* y) {
  const int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
  return a > b ? -1 : (a < b);
}

/* ---------------------------------------------------------------------------------------- */
/* Compression.                                                                               */
/* ---------------------------------------------------------------------------------------- */
#define NC_COMPRESS(T, SUFFIX)                                                                   \
  static int compress_##SUFFIX(const T* prev, const T* cur, int64_t n, int B, double E,         \
                               int anchor, int64_t block_bytes, int threads, unsigned char* out, \
                               size_t cap, size_t* out_size) {                                   \
    const int L = (int)sizeof(T);                                                                \
    const int dtype = L == 8;                                                                    \
    pass1_##SUFFIX c1;                                                                           \
    memset(&c1, 0, sizeof(c1));                                                                  \
    c1.prev = prev;                                                                              \
    c1.cur = cur;                                                                                \
    c1.E_T = (T)E;                                                                               \
    c1.w = c1.E_T + c1.E_T;                                                                      \
    c1.inv_w = (T)1 / c1.w;                                                                      \
    c1.cap = c1.w * (T)(1 << NC_WIN_LOG2);                                                       \
    int rc = NC_OK;                                                                              \
    T mins[256];                                                                                 \
    int anys[256];                                                                               \
    int64_t tmin[256], tmax[256];                                                                \
    if (threads < 1) threads = 1;                                                                \
    if (threads > 256) threads = 256;                                                            \
    /* grid origin (reading R2): -E, or the smallest binnable ratio (+0 for a zero minimum) */   \
    if (anchor == 0) {                                                                           \
      c1.a = -c1.E_T;                                                                            \
      c1.hbase = -((int64_t)1 << NC_WIN_LOG2) - NC_MARGIN;                                       \
    } else {                                                                                     \
      c1.minr = mins;                                                                            \
      c1.anyr = anys;                                                                            \
      if ((rc = parallel_for(threads, n, min_body_##SUFFIX, &c1))) return rc;                    \
      int any = 0;                                                                               \
      T a = 0;                                                                                   \
      for (int i = 0; i < threads; ++i)                                                          \
        if (anys[i] && (!any || mins[i] < a)) { a = mins[i]; any = 1; }                          \
      c1.a = (any && a != 0) ? a : (T)0;                                                         \
      c1.hbase = -NC_MARGIN;                                                                     \
    }                                                                                            \
    c1.bins = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));                       \
    c1.hist = (uint32_t*)calloc((size_t)threads * NC_HBINS, sizeof(uint32_t));                   \
    if (!c1.bins || !c1.hist) { free(c1.bins); free(c1.hist); return NC_ENOMEM; }                \
    c1.tmin = tmin;                                                                              \
    c1.tmax = tmax;                                                                              \
    for (int i = 0; i < threads; ++i) { tmin[i] = INT64_MAX; tmax[i] = INT64_MIN; }              \
    if ((rc = parallel_for(threads, n, bin_body_##SUFFIX, &c1)) || c1.err) {                     \
      free(c1.bins); free(c1.hist); return rc ? rc : NC_EINVAL;                                  \
    }                                                                                            \
    /* merged histogram over the bin range seen (the paper's MPI_Allreduce) */                  \
    int64_t bmin = INT64_MAX, bmax = INT64_MIN;                                                  \
    for (int i = 0; i < threads; ++i) {                                                          \
      if (tmin[i] < bmin) bmin = tmin[i];                                                        \
      if (tmax[i] > bmax) bmax = tmax[i];                                                        \
    }                                                                                            \
    const int64_t R = bmax >= bmin ? bmax - bmin + 1 : 0;                                        \
    bc_t* nz = (bc_t*)malloc((size_t)(R > 0 ? R : 1) * sizeof(bc_t));                           \
    int64_t nnz = 0;                                                                             \
    for (int64_t k = 0; k < R; ++k) {                                                            \
      int64_t s = 0;                                                                             \
      for (int i = 0; i < threads; ++i) s += c1.hist[(size_t)i * NC_HBINS + (bmin + k - c1.hbase)]; \
      if (s) { nz[nnz].bin = bmin + k; nz[nnz].count = s; ++nnz; }                               \
    }                                                                                            \
    free(c1.hist);                                                                               \
    /* automatic index length (§IV.B.2, Eqs. 5 and 6, reading R10) */                            \
    if (B == 0) {                                                                                \
      int64_t* desc = (int64_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));           \
      for (int64_t i = 0; i < nnz; ++i) desc[i] = nz[i].count;                                   \
      qsort(desc, (size_t)nnz, sizeof(int64_t), by_count_desc);                                  \
      int64_t best_bits = 0, top = 0, used = 0;                                                  \
      for (int b = 1; b <= 16; ++b) {                                                            \
        const int64_t kk = ((int64_t)1 << b) - 1;                                                \
        while (used < kk && used < nnz) top += desc[used++];                                     \
        const int64_t bits = 8 * ((int64_t)1 << b) * L + n * b + 8 * (int64_t)L * (n - top);     \
        if (b == 1 || bits < best_bits) { best_bits = bits; B = b; }                             \
      }                                                                                          \
      free(desc);                                                                                \
    }                                                                                            \
    const layout_t g = make_layout(n, L, B, block_bytes);                                        \
    if (cap < (size_t)(g.off_exact + n * L)) { free(nz); free(c1.bins); return NC_ECAP; }        \
    /* top-k selection (§IV.B.1): count descending, ties to the smaller bin; ranks ascending */   \
    const int64_t kk = ((int64_t)1 << B) - 1;                                                    \
    qsort(nz, (size_t)nnz, sizeof(bc_t), by_count_then_bin);                                     \
    const int64_t n_sel = nnz < kk ? nnz : kk;                                                   \
    qsort(nz, (size_t)n_sel, sizeof(bc_t), by_bin);                                              \
    T* mult = (T*)malloc(((size_t)1 << B) * sizeof(T));                                          \
    int32_t* rank = (int32_t*)malloc((size_t)(R > 0 ? R : 1) * sizeof(int32_t));                 \
    uint8_t* marker = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));                                 \
    int64_t* tile_count = (int64_t*)malloc((size_t)(g.nsub + 1) * sizeof(int64_t));             \
    if (!mult || !rank || !marker || !tile_count) {                                              \
      free(mult); free(rank); free(marker); free(tile_count); free(nz); free(c1.bins);           \
      return NC_ENOMEM;                                                                          \
    }                                                                                            \
    memset(out, 0, (size_t)g.off_exact);                                                         \
    T* centres = (T*)malloc(((size_t)1 << B) * sizeof(T));                                       \
    for (int64_t r = 0; r < ((int64_t)1 << B); ++r) {                                            \
      T cr = 0;                                                                                  \
      if (r < n_sel) cr = c1.a + (((T)nz[r].bin + (T)0.5) * c1.w);   /* centre (reading R6) */  \
      centres[r] = cr;                                                                           \
      mult[r] = (T)1 + cr;                                                                       \
    }                                                                                            \
    memcpy(out + g.off_centres, centres, ((size_t)1 << B) * sizeof(T));                          \
    free(centres);                                                                               \
    for (int64_t k = 0; k < R; ++k) rank[k] = -1;                                                \
    for (int64_t r = 0; r < n_sel; ++r) rank[nz[r].bin - bmin] = (int32_t)r;                     \
    free(nz);                                                                                    \
    pass2_##SUFFIX c2;                                                                           \
    c2.prev = prev;                                                                              \
    c2.cur = cur;                                                                                \
    c2.bins = c1.bins;                                                                           \
    c2.rank = rank;                                                                              \
    c2.rbase = bmin;                                                                             \
    c2.rlen = R;                                                                                 \
    c2.mult = mult;                                                                              \
    c2.E_T = c1.E_T;                                                                             \
    c2.g = g;                                                                                    \
    c2.blob = out;                                                                               \
    c2.marker = marker;                                                                          \
    c2.tile_count = tile_count;                                                                  \
    rc = parallel_for(threads, g.nsub, assign_body_##SUFFIX, &c2);                               \
    free(c1.bins);                                                                               \
    free(rank);                                                                                  \
    free(mult);                                                                                  \
    if (rc) { free(marker); free(tile_count); return rc; }                                       \
    /* offsets (§IV.C): sub-block table, per-block table, index-block starts */                  \
    int64_t* sub_off = (int64_t*)(void*)(out + g.off_sub_off);                                   \
    int64_t* inc_off = (int64_t*)(void*)(out + g.off_inc_off);                                   \
    int64_t* idx_off = (int64_t*)(void*)(out + g.off_idx_off);                                   \
    const int64_t spb = cdiv(g.epb, NC_SUB);                                                     \
    int64_t run = 0;                                                                             \
    for (int64_t gt = 0; gt < g.nsub; ++gt) {                                                    \
      int64_t v = run;                                                                           \
      memcpy(&sub_off[gt], &v, 8);                                                               \
      if (gt % spb == 0) memcpy(&inc_off[gt / spb], &v, 8);                                      \
      run += tile_count[gt];                                                                     \
      tile_count[gt] = v;                                                                        \
    }                                                                                            \
    memcpy(&inc_off[g.nblocks], &run, 8);                                                        \
    for (int64_t q = 0; q <= g.nblocks; ++q) {                                                   \
      const int64_t v = q < g.nblocks ? q * g.block_stride : g.index_bytes;                      \
      memcpy(&idx_off[q], &v, 8);                                                                \
    }                                                                                            \
    const int64_t n_inc = run;                                                                   \
    pass3_##SUFFIX c3;                                                                           \
    c3.cur = cur;                                                                                \
    c3.marker = marker;                                                                          \
    c3.tile_off = tile_count;                                                                    \
    c3.g = g;                                                                                    \
    c3.exact = (T*)(void*)(out + g.off_exact);                                                   \
    rc = parallel_for(threads, g.nsub, exact_body_##SUFFIX, &c3);                                \
    free(marker);                                                                                \
    free(tile_count);                                                                            \
    if (rc) return rc;                                                                           \
    write_header(out, &g, dtype, E, anchor, block_bytes, n_sel, n_inc, (double)c1.a);            \
    *out_size = (size_t)(g.off_exact + n_inc * L);                                               \
    return NC_OK;                                                                                \
  }

NC_COMPRESS(float, f32)
NC_COMPRESS(double, f64)

int ncpu_compress(const void* prev, const void* cur, int64_t n, int dtype, int B, double E,
                  int anchor, int64_t block_bytes, int threads, void* out, size_t cap,
                  size_t* out_size) {
  if (n < 0 || (n > 0 && (!prev || !cur)) || !out || !out_size) return NC_EINVAL;
  if (B < 0 || B > 16 || !(E > 0 && E < 1) || (anchor != 0 && anchor != 1) || block_bytes < 2)
    return NC_EINVAL;
  if (dtype)
    return compress_f64((const double*)prev, (const double*)cur, n, B, E, anchor, block_bytes,
                        threads, (unsigned char*)out, cap, out_size);
  return compress_f32((const float*)prev, (const float*)cur, n, B, E, anchor, block_bytes,
                      threads, (unsigned char*)out, cap, out_size);
}

/* ---------------------------------------------------------------------------------------- */
/* Decompression (§III.E).                                                                    */
/* ---------------------------------------------------------------------------------------- */
static int64_t get64(const unsigned char* p) { int64_t v; memcpy(&v, p, 8); return v; }
static int32_t get32(const unsigned char* p) { int32_t v; memcpy(&v, p, 4); return v; }

int ncpu_decompress(const void* blob, size_t size, const void* prev, void* out, int64_t n,
                    int threads) {
  const unsigned char* b = (const unsigned char*)blob;
  if (!b || size < NC_HEADER) return NC_EINVAL;
  if ((uint32_t)get32(b) != NC_MAGIC || (uint32_t)get32(b + 4) != NC_VERSION) return NC_ECORRUPT;
  const int dtype = get32(b + 8), B = get32(b + 12);
  if (B < 1 || B > 16 || (dtype != 0 && dtype != 1) || get64(b + 32) != n) return NC_EINVAL;
  const layout_t g = make_layout(n, dtype ? 8 : 4, B, get64(b + 40));
  const int64_t n_inc = get64(b + 88);
  if (g.off_exact != get64(b + 152) || (size_t)(g.off_exact + n_inc * g.L) > size) return NC_ECORRUPT;
  int rc, err;
  if (dtype) {
    double* mult = (double*)malloc(((size_t)1 << B) * sizeof(double));
    if (!mult) return NC_ENOMEM;
    const double* c = (const double*)(const void*)(b + g.off_centres);
    for (int r = 0; r < (1 << B); ++r) mult[r] = 1.0 + c[r];
    pass4_f64 c4 = {(const double*)prev, (double*)out, b, g,
                    (const int64_t*)(const void*)(b + g.off_sub_off), mult,
                    (const double*)(const void*)(b + g.off_exact), n_inc, 0};
    rc = parallel_for(threads, g.nsub, decode_body_f64, &c4);
    err = c4.err;
    free(mult);
  } else {
    float* mult = (float*)malloc(((size_t)1 << B) * sizeof(float));
    if (!mult) return NC_ENOMEM;
    const float* c = (const float*)(const void*)(b + g.off_centres);
    for (int r = 0; r < (1 << B); ++r) mult[r] = 1.0f + c[r];
    pass4_f32 c4 = {(const float*)prev, (float*)out, b, g,
                    (const int64_t*)(const void*)(b + g.off_sub_off), mult,
                    (const float*)(const void*)(b + g.off_exact), n_inc, 0};
    rc = parallel_for(threads, g.nsub, decode_body_f32, &c4);
    err = c4.err;
    free(mult);
  }
  return rc ? rc : (err ? NC_ECORRUPT : NC_OK);
}
