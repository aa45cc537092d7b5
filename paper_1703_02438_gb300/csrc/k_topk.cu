// k_topk.cu — K2: top-k bin selection over the global histogram (§IV.B.1), centre table
// (§III.B), multipliers for the assignment pass, and the blob header (§IV.D, Fig. 2).
//
// The paper runs the top-k selection serially and replicated on every rank (§IV.B.1, it takes
// under 1.5% of the binning phase, Table 3). Here one CTA of 1024 threads does it on the
// device: a radix select finds the k-th largest count T, then an ordered scan over the bin
// range takes every bin with count > T and the lowest-numbered bins with count == T
// (ties go to the smaller bin id), and a second scan numbers the selected bins in ascending
// bin order. The CTA also restores the workspace invariant (histogram and keys back to 0).
//
// k2_auto_b, for B = 0, chooses the index length from the same histogram before K2 runs
// (§IV.B.2, Eqs. 5 and 6); it only reads the histogram.
#include "launch.h"

namespace nmk {

namespace {

constexpr int K2_THREADS = 1024;
constexpr int K2_ITEMS = 4;

struct TopkArgs {
  Ctrl* ctrl;
  unsigned long long* hist;
  unsigned short* rank_of;
  int* selb;
  unsigned char* blob;
  void* mtab;
  float* cftab;
  Geometry g;
  numarck_header hdr;
};

// Exclusive block scan of one int per thread (1024 threads). s must hold 33 ints.
__device__ __forceinline__ int block_excl_scan(int v, int* s, int& total) {
  const int lane = (int)lane_id(), w = (int)(threadIdx.x >> 5);
  const int inc = warp_incl_scan(v);
  if (lane == 31) s[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int t = s[lane];
    const int ti = warp_incl_scan(t);
    s[lane] = ti - t;
    if (lane == 31) s[32] = ti;
  }
  __syncthreads();
  const int ex = s[w] + inc - v;
  total = s[32];
  __syncthreads();
  return ex;
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* s) {
  const int lane = (int)lane_id(), w = (int)(threadIdx.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s[w] = v;
  __syncthreads();
  if (w == 0) {
    long long t = s[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s[32] = t;
  }
  __syncthreads();
  const long long r = s[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned long long block_max_ull(unsigned long long v,
                                                            unsigned long long* s) {
  const int lane = (int)lane_id(), w = (int)(threadIdx.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  if (lane == 0) s[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = s[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, t, o);
      t = u > t ? u : t;
    }
    if (lane == 0) s[32] = t;
  }
  __syncthreads();
  const unsigned long long r = s[32];
  __syncthreads();
  return r;
}

// k-th largest of the non-zero values H[0..R) (k >= 1, more than k non-zero values, mx = the
// largest value): *thr = that value and *need = how many values equal to it the k largest
// include. Radix select, 8 bits per pass from the top bit of mx; called by all K2_THREADS.
__device__ __forceinline__ void select_kth_largest(const unsigned long long* H, int R, long long k,
                                                   unsigned long long mx, unsigned int* s_dig,
                                                   unsigned long long* s_prefix,
                                                   long long* s_rem, unsigned long long* thr,
                                                   long long* need) {
  const int tid = (int)threadIdx.x;
  const int top = 63 - __clzll((long long)mx);
  unsigned long long prefix = 0;
  long long rem = k;
  for (int shift = (top / 8) * 8; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += K2_THREADS) s_dig[i] = 0u;
    __syncthreads();
    for (int i = tid; i < R; i += K2_THREADS) {
      const unsigned long long v = H[i];
      if (v != 0 && (shift + 8 >= 64 || (v >> (shift + 8)) == (prefix >> (shift + 8))))
        atomicAdd(&s_dig[(v >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      long long cum = 0;
      for (int d = 255; d >= 0; --d) {
        if (cum + (long long)s_dig[d] >= rem) {
          *s_prefix = prefix | ((unsigned long long)d << shift);
          *s_rem = rem - cum;
          break;
        }
        cum += s_dig[d];
      }
    }
    __syncthreads();
    prefix = *s_prefix;
    rem = *s_rem;
    __syncthreads();
  }
  *thr = prefix;
  *need = rem;
}

// Automatic index length (§IV.B.2, Eqs. 5 and 6), one CTA after K1: for B = 1..16 the
// compressible points are those in the top k = 2^B - 1 bins of the histogram, alpha(B) =
// (n - compressible) / n, and 8 * file_size(B) = 8 * 2^B * L + n * B + 8 * L * n * alpha(B)
// (exact integers); the smallest wins (ties: smaller B) and is written to ctrl->auto_B. The sum
// of the top k counts for every k <= 65535 follows from the counts above the 65535-th largest
// (compacted into `list`, fewer than 65535 of them) plus copies of that count.
struct AutoArgs {
  Ctrl* ctrl;
  const unsigned long long* hist;
  unsigned long long* list;     // scratch, 65536 entries
  int hbase;
  long long n;
  int L;
};

__global__ void __launch_bounds__(K2_THREADS, 1) k2_auto_b(AutoArgs A) {
  __shared__ long long s_ll[33];
  __shared__ unsigned long long s_ull[33];
  __shared__ unsigned int s_dig[256];
  __shared__ unsigned long long s_prefix;
  __shared__ long long s_rem;
  __shared__ int s_m;
  Ctrl* ctrl = A.ctrl;
  const int tid = (int)threadIdx.x;
  const unsigned kmin = ctrl->bmin_key, kmax = ctrl->bmax_key;
  const int any = kmax != 0u;
  const int bmin = any ? (int)(KEY_BIAS - kmin) : 0;
  const int bmax = any ? (int)(kmax - KEY_BIAS) : -1;
  int R = bmax - bmin + 1;
  const int i0 = bmin - A.hbase;
  if (any && (i0 < 0 || i0 + R > HWIN || ctrl->win_err)) R = 0;   // K2 reports the error
  const unsigned long long* H = A.hist + (any ? i0 : 0);
  constexpr long long KTOP = (1LL << NUMARCK_MAX_B) - 1;

  long long nnz = 0;
  unsigned long long mx = 0;
  for (int i = tid; i < R; i += K2_THREADS) {
    const unsigned long long v = H[i];
    nnz += v != 0;
    mx = v > mx ? v : mx;
  }
  nnz = block_sum_ll(nnz, s_ll);
  mx = block_max_ull(mx, s_ull);
  unsigned long long tmax = 0;   // the KTOP-th largest count (0 when at most KTOP bins)
  long long need_max = 0;
  if (nnz > KTOP) select_kth_largest(H, R, KTOP, mx, s_dig, &s_prefix, &s_rem, &tmax, &need_max);
  if (tid == 0) s_m = 0;
  __syncthreads();
  for (int i = tid; i < R; i += K2_THREADS) {
    const unsigned long long v = H[i];
    if (v > tmax) A.list[atomicAdd(&s_m, 1)] = v;
  }
  __syncthreads();
  const int m = s_m;                               // counts above tmax (fewer than KTOP)
  unsigned long long lmx = 0;
  long long lsum = 0;
  for (int i = tid; i < m; i += K2_THREADS) {
    lsum += (long long)A.list[i];
    lmx = A.list[i] > lmx ? A.list[i] : lmx;
  }
  lsum = block_sum_ll(lsum, s_ll);
  lmx = block_max_ull(lmx, s_ull);
  const long long n = A.n, L = A.L;
  long long best_bits = -1;
  int best_B = 1;
  for (int B = 1; B <= NUMARCK_MAX_B; ++B) {
    const long long k = (1LL << B) - 1;
    long long cov;
    if (k >= m) {
      cov = lsum + (k - m) * (long long)tmax;      // k - m <= need_max copies of tmax
    } else {
      unsigned long long t = 0;
      long long need = 0;
      select_kth_largest(A.list, m, k, lmx, s_dig, &s_prefix, &s_rem, &t, &need);
      long long above = 0;
      for (int i = tid; i < m; i += K2_THREADS) above += A.list[i] > t ? (long long)A.list[i] : 0;
      cov = block_sum_ll(above, s_ll) + need * (long long)t;
    }
    const long long bits = 8 * (1LL << B) * L + n * B + 8 * L * (n - cov);
    if (best_bits < 0 || bits < best_bits) {
      best_bits = bits;
      best_B = B;
    }
  }
  (void)need_max;
  if (tid == 0) ctrl->auto_B = best_B;
}

template <typename T>
__device__ __forceinline__ T anchor_value(const Ctrl* ctrl, const Consts<T>& c, int anchor) {
  if (anchor != NUMARCK_ANCHOR_MIN) return c.a;
  const unsigned long long key = ctrl->amin_key;
  double a = key ? key_to_ratio(key) : 0.0;
  if (a == 0.0) a = 0.0;
  return (T)a;
}

template <typename T>
__device__ __forceinline__ void k2_body(const TopkArgs& A, const Consts<T>& c) {
  __shared__ int s_scan[33];
  __shared__ long long s_ll[33];
  __shared__ unsigned long long s_ull[33];
  __shared__ unsigned int s_dig[256];
  __shared__ unsigned long long s_prefix;
  __shared__ long long s_rem;

  Ctrl* ctrl = A.ctrl;
  const Geometry& g = A.g;
  const int tid = (int)threadIdx.x;
  const unsigned kmin = ctrl->bmin_key, kmax = ctrl->bmax_key;
  const int any = kmax != 0u;
  const int bmin = any ? (int)(KEY_BIAS - kmin) : 0;
  const int bmax = any ? (int)(kmax - KEY_BIAS) : -1;
  const T a = anchor_value<T>(ctrl, c, g.anchor);
  int R = bmax - bmin + 1;
  const int i0 = bmin - c.hbase;
  int status = 0;
  // On a window error the selection is skipped (R = 0), but K1 has still counted the bins that
  // fell inside the window: [clr_lo, clr_hi) is that range, cleared below so that a failed call
  // leaves the workspace ready like any other.
  int clr_lo = 0, clr_hi = 0;
  if (any && (i0 < 0 || i0 + R > HWIN || ctrl->win_err)) {
    status = NUMARCK_ERR_CORRUPT;
    clr_lo = i0 > 0 ? i0 : 0;
    clr_hi = bmax - c.hbase + 1 < HWIN ? bmax - c.hbase + 1 : HWIN;
    R = 0;
  }
  // an error of the decompression that made this compression's prev (fused step) marks the blob
  if (ctrl->error) status = ctrl->error;
  unsigned long long* H = A.hist + (any ? i0 : 0);
  const int k = (1 << g.B) - 1;
  const int M = g.M;

  // pass 1: non-empty bins and the largest count
  long long nnz = 0;
  unsigned long long mx = 0;
  for (int i = tid; i < R; i += K2_THREADS) {
    const unsigned long long v = H[i];
    nnz += v != 0;
    mx = v > mx ? v : mx;
  }
  nnz = block_sum_ll(nnz, s_ll);
  mx = block_max_ull(mx, s_ull);

  // radix select of the k-th largest count (when more than k bins are non-empty)
  unsigned long long thr = 0;  // select count > thr, plus `need` bins with count == thr
  long long need = 0;
  if (nnz > k) select_kth_largest(H, R, k, mx, s_dig, &s_prefix, &s_rem, &thr, &need);

  // ordered scans over the bin range: ties in count go to the smaller bin, then ranks
  int tie_base = 0, rank_base = 0;
  for (int base = 0; base < R; base += K2_THREADS * K2_ITEMS) {
    const int i = base + tid * K2_ITEMS;
    unsigned long long cc[K2_ITEMS];
    int tie_l = 0;
#pragma unroll
    for (int it = 0; it < K2_ITEMS; ++it) {
      cc[it] = (i + it < R) ? H[i + it] : 0ull;
      tie_l += (i + it < R && cc[it] == thr) ? 1 : 0;
    }
    int tie_tot = 0;
    int tr = tie_base + block_excl_scan(tie_l, s_scan, tie_tot);
    bool sf[K2_ITEMS];
    int sel_l = 0;
#pragma unroll
    for (int it = 0; it < K2_ITEMS; ++it) {
      const bool in = i + it < R;
      const bool tie = in && cc[it] == thr;
      sf[it] = in && (cc[it] > thr || (tie && tr < need));
      tr += tie ? 1 : 0;
      sel_l += sf[it] ? 1 : 0;
    }
    int sel_tot = 0;
    int r = rank_base + block_excl_scan(sel_l, s_scan, sel_tot);
#pragma unroll
    for (int it = 0; it < K2_ITEMS; ++it) {
      if (i + it < R) {
        A.rank_of[i0 + i + it] = (unsigned short)(sf[it] ? r : M);
        if (sf[it]) A.selb[r] = bmin + i + it;
        r += sf[it] ? 1 : 0;
      }
    }
    tie_base += tie_tot;
    rank_base += sel_tot;
  }
  const int n_sel = rank_base;
  __syncthreads();

  // centres (blob), multipliers m = 1 + centre and float32 copies of m - 1 (workspace)
  T* centres = reinterpret_cast<T*>(A.blob + g.off_centres);
  T* mt = reinterpret_cast<T*>(A.mtab);
  for (int r = tid; r < (1 << g.B); r += K2_THREADS) {
    T cr = (T)0, m = (T)1;
    if (r < n_sel) {
      cr = bin_centre<T>(A.selb[r], a, c.w);
      m = t_add((T)1, cr);
    }
    centres[r] = cr;
    mt[r] = m;
    A.cftab[r] = (float)t_sub(m, (T)1);
  }

  // restore the zero state of the histogram range and the keys
  for (int i = tid; i < R; i += K2_THREADS) H[i] = 0ull;
  for (int i = clr_lo + tid; i < clr_hi; i += K2_THREADS) A.hist[i] = 0ull;

  // blob: idx_off (closed form), the zero gaps between sections, the header
  int64_t* idx_off = reinterpret_cast<int64_t*>(A.blob + g.off_idx_off);
  for (int64_t q = tid; q <= g.nblocks; q += K2_THREADS)
    idx_off[q] = q < g.nblocks ? q * g.block_stride : g.index_bytes;
  int64_t* inc_off = reinterpret_cast<int64_t*>(A.blob + g.off_inc_off);
  if (tid == 0) inc_off[g.nblocks] = 0;  // final value written by K3 when n > 0
  const int L = g.dtype == NUMARCK_F64 ? 8 : 4;
  const int64_t gaps[5][2] = {
      {g.off_centres + ((int64_t)1 << g.B) * L, g.off_idx_off},
      {g.off_idx_off + (g.nblocks + 1) * 8, g.off_inc_off},
      {g.off_inc_off + (g.nblocks + 1) * 8, g.off_sub_off},
      {g.off_sub_off + g.nsub * 8, g.off_index},
      {g.off_index + g.index_bytes, g.off_exact}};
#pragma unroll
  for (int s = 0; s < 5; ++s)
    for (int64_t o = gaps[s][0] + tid; o < gaps[s][1]; o += K2_THREADS) A.blob[o] = 0;

  __syncthreads();
  if (tid == 0) {
    numarck_header h = A.hdr;
    h.n_sel = n_sel;
    h.a = (double)a;
    h.status = status;
    const uint4* src = reinterpret_cast<const uint4*>(&h);
    uint4* dst = reinterpret_cast<uint4*>(A.blob);
#pragma unroll
    for (int i = 0; i < NUMARCK_HEADER_BYTES / 16; ++i) dst[i] = src[i];
    ctrl->bmin_key = 0u;
    ctrl->bmax_key = 0u;
    ctrl->amin_key = 0ull;
    ctrl->win_err = 0u;
    ctrl->error = 0;
    ctrl->any = any && R > 0;
    ctrl->sel_bmin = bmin;
    ctrl->sel_bmax = bmax;
    ctrl->sel_lo = n_sel > 0 ? A.selb[0] : 1;            // ranks follow ascending bin order
    ctrl->sel_hi = n_sel > 0 ? A.selb[n_sel - 1] : 0;
    ctrl->n_sel = n_sel;
    ctrl->a = (double)a;
  }
}

template <typename T>
__global__ void __launch_bounds__(K2_THREADS, 1) k2_topk(TopkArgs A, Consts<T> c) {
  k2_body<T>(A, c);
}

// Fused batch (K6): K2 of every variable of a batch in one launch, CTA v for variable v.
__global__ void __launch_bounds__(K2_THREADS, 1) k2_fused(FusedArgs F) {
  const FusedVar& V = F.vars[blockIdx.x];
  TopkArgs A;
  A.ctrl = reinterpret_cast<Ctrl*>(V.ws + V.wl.ctrl);
  A.hist = reinterpret_cast<unsigned long long*>(V.ws + V.wl.hist);
  A.rank_of = reinterpret_cast<unsigned short*>(V.ws + V.wl.rank);
  A.selb = reinterpret_cast<int*>(V.ws + V.wl.selb);
  A.blob = V.blob;
  A.mtab = V.ws + V.wl.mtab;
  A.cftab = reinterpret_cast<float*>(V.ws + V.wl.cftab);
  A.g = V.g;
  A.hdr = make_header(V.g, V.E, V.block_bytes);
  if (V.g.dtype == NUMARCK_F64)
    k2_body<double>(A, V.cd);
  else
    k2_body<float>(A, V.cf);
}

}  // namespace

cudaError_t launch_auto_b(const CompressPlan& P, cudaStream_t s) {
  AutoArgs A;
  A.ctrl = reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl);
  A.hist = reinterpret_cast<const unsigned long long*>(P.ws + P.wl.hist);
  A.list = reinterpret_cast<unsigned long long*>(P.ws + P.wl.mtab);   // filled by K2 later
  A.hbase = P.g.dtype == NUMARCK_F64 ? P.cd.hbase : P.cf.hbase;
  A.n = P.g.n;
  A.L = P.g.dtype == NUMARCK_F64 ? 8 : 4;
  k2_auto_b<<<1, K2_THREADS, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_topk(const CompressPlan& P, cudaStream_t s) {
  TopkArgs A;
  A.ctrl = reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl);
  A.hist = reinterpret_cast<unsigned long long*>(P.ws + P.wl.hist);
  A.rank_of = reinterpret_cast<unsigned short*>(P.ws + P.wl.rank);
  A.selb = reinterpret_cast<int*>(P.ws + P.wl.selb);
  A.blob = P.blob;
  A.mtab = P.ws + P.wl.mtab;
  A.cftab = reinterpret_cast<float*>(P.ws + P.wl.cftab);
  A.g = P.g;
  A.hdr = P.hdr;
  if (P.g.dtype == NUMARCK_F64)
    k2_topk<double><<<1, K2_THREADS, 0, s>>>(A, P.cd);
  else
    k2_topk<float><<<1, K2_THREADS, 0, s>>>(A, P.cf);
  return cudaGetLastError();
}

cudaError_t launch_fused_topk(const FusedArgs& F, cudaStream_t s) {
  if (F.count <= 0) return cudaSuccess;
  k2_fused<<<F.count, K2_THREADS, 0, s>>>(F);
  return cudaGetLastError();
}

}  // namespace nmk
