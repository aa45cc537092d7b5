// k1.cuh — the per-point step of K1 (change ratio, bin, own-bin check, histogram, code), shared
// by the histogram kernel (k_hist.cu) and the fused decompress-and-classify kernel (k_step.cu).
//
// Method steps: Eq. 1 change ratio, §IV.B.1 bin ids and histogram, §III.C error-bound check
// against the centre of the point's own bin (the only centre it can be indexed to).
#pragma once

#include "launch.h"

namespace nmk {

struct HistCtx {
  unsigned int* sh;
  unsigned long long* hist;
  Ctrl* ctrl;
  int sbase;
  int hbase;
  int cbase;                  // bin of code 0
  unsigned short* codes;      // per-element bin codes (scratch at the blob's tail)
};

__device__ __forceinline__ unsigned bin_code(const HistCtx& h, bool binned, int b, bool pass) {
  if (!binned) return CODE_NONE;
  const unsigned off = (unsigned)(b - h.cbase);
  return off < (unsigned)CODE_BINS ? (off << 1) | (pass ? 1u : 0u) : CODE_FAR;
}

// One point of bin b into the histogram (if valid): a shared-memory atomic inside the shared
// window (the hardware resolves lanes of a warp that hit the same bin; measured faster here
// than aggregating them first with match.any, on concentrated and on spread bins alike), a
// global one outside it. Bins outside the shared window also update this thread's bin range
// (the range of the bins inside it is read from the shared histogram at the end).
__device__ __forceinline__ void hist_add(const HistCtx& h, bool valid, int b, int& lmin,
                                         int& lmax) {
  if (!valid) return;
  const int si = b - h.sbase;
  if ((unsigned)si < (unsigned)SH_BINS) {
    atomicAdd(&h.sh[si], 1u);
  } else {
    lmin = min(lmin, b);
    lmax = max(lmax, b);
    const int gi = b - h.hbase;
    if ((unsigned)gi < (unsigned)HWIN)
      atomicAdd(&h.hist[gi], 1ull);
    else
      atomicOr(&h.ctrl->win_err, 1u);
  }
}

// Exact bin and own-bin check (§III.B, §III.C) of one float64 point (the rare undecided points).
static __device__ __noinline__ int classify_check_f64_slow(double p, double x,
                                                           const Consts<double>& c, int cbase,
                                                           int* b, bool* pass) {
  int bb = 0;
  const int k = classify_exact<double>(p, x, c, bb);
  *b = bb;
  *pass = k && (unsigned)(bb - cbase) < (unsigned)CODE_BINS &&
          check_exact<double>(p, x, bin_multiplier<double>(bb, c.a, c.w), c.E_T);
  return k;
}

template <typename T>
struct Classifier;

// fast(): 0 (not binnable), 1 (bin in b; pass = the own-bin check when b is in the code window)
// or 2/3 (undecided: call exact()). exact() decides both with the exact T sequences.
// (ZERO_P: the float64 estimate decides p = +-0 itself rather than leaving it to exact(); K1 takes
// it, K41 does not: there the test cost more issue slots than the queued zeros.)
template <>
struct Classifier<float> {
  template <bool ZERO_P = true>
  __device__ __forceinline__ static int fast(float p, float x, const Consts<float>& c, int cbase,
                                             int& b, bool& pass) {
    return exact(p, x, c, cbase, b, pass);
  }
  __device__ __forceinline__ static int exact(float p, float x, const Consts<float>& c, int cbase,
                                              int& b, bool& pass) {
    const int k = classify_exact<float>(p, x, c, b);
    pass = k && (unsigned)(b - cbase) < (unsigned)CODE_BINS &&
           check_exact<float>(p, x, bin_multiplier<float>(b, c.a, c.w), c.E_T);
    return k;
  }
};
template <>
struct Classifier<double> {
  template <bool ZERO_P = true>
  __device__ __forceinline__ static int fast(double p, double x, const Consts<double>& c,
                                             int cbase, int& b, bool& pass) {
    return classify_check_f64_fast<ZERO_P>(p, x, c, cbase, b, pass);
  }
  __device__ static int exact(double p, double x, const Consts<double>& c, int cbase, int& b,
                              bool& pass) {
    return classify_check_f64_slow(p, x, c, cbase, &b, &pass);
  }
};

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  using codes = uint2;   // 4 codes
  static constexpr int N = 4;
  __device__ __forceinline__ static void get(const type& v, float* o) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ __forceinline__ static codes pack(const unsigned* k) {
    return make_uint2(k[0] | (k[1] << 16), k[2] | (k[3] << 16));
  }
};
template <>
struct Vec<double> {
  using type = double2;
  using codes = unsigned;   // 2 codes
  static constexpr int N = 2;
  __device__ __forceinline__ static void get(const type& v, double* o) {
    o[0] = v.x; o[1] = v.y;
  }
  __device__ __forceinline__ static codes pack(const unsigned* k) { return k[0] | (k[1] << 16); }
};


// Start of a K1 pass (every CTA; ends with a block barrier): clears this CTA's shared window,
// and (grid-wide) the next compression's per-tile counts, offset-scan flags and scan ticket;
// CTA 0 publishes the bin of code 0.
__device__ __forceinline__ void k1_begin(const HistCtx& h, unsigned long long* tstatus,
                                         int64_t nsub) {
  if (blockIdx.x == 0 && threadIdx.x == 0) h.ctrl->code_base = h.cbase;
  for (int i = threadIdx.x; i < SH_BINS; i += blockDim.x) h.sh[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) h.ctrl->ticket = 0u;
  const int64_t nstat = nsub > 0 ? nsub + nsub / 4096 + 2 : 0;   // counts + scan flags
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nstat;
       i += (int64_t)gridDim.x * blockDim.x)
    tstatus[i] = 0ull;
  __syncthreads();
}

// End of a K1 pass (every thread of the CTA): merges the shared window into the global
// histogram; the bins it holds and this thread's out-of-window range (lmin, lmax) give the
// CTA's bin range, folded into the global range keys with one atomic each.
__device__ __forceinline__ void k1_end(const HistCtx& h, int lmin, int lmax) {
  __shared__ int s_min, s_max;
  if (threadIdx.x == 0) { s_min = 0x7FFFFFFF; s_max = (int)0x80000000; }
  __syncthreads();   // every shared-histogram update is done
  for (int i = threadIdx.x; i < SH_BINS; i += blockDim.x) {
    const unsigned v = h.sh[i];
    if (v) {
      const int b = h.sbase + i;
      lmin = min(lmin, b);
      lmax = max(lmax, b);
      const int gi = b - h.hbase;
      if ((unsigned)gi < (unsigned)HWIN)
        atomicAdd(&h.hist[gi], (unsigned long long)v);
      else
        atomicOr(&h.ctrl->win_err, 1u);
    }
  }
  lmin = __reduce_min_sync(0xffffffffu, lmin);
  lmax = __reduce_max_sync(0xffffffffu, lmax);
  if (lane_id() == 0 && lmin <= lmax) { atomicMin(&s_min, lmin); atomicMax(&s_max, lmax); }
  __syncthreads();
  if (threadIdx.x == 0 && s_min <= s_max) {
    atomicMax(&h.ctrl->bmin_key, KEY_BIAS - (unsigned)s_min);
    atomicMax(&h.ctrl->bmax_key, (unsigned)s_max + KEY_BIAS);
  }
}


// ---------------------------------------------------------------------------------------
// The loops of K0 and K1 over a range of one variable, shared by the single-variable kernels
// (k_hist.cu: the whole variable, a grid-stride loop) and the fused batch kernels (k_fused.cu:
// a CTA's contiguous part of each variable it covers).
// ---------------------------------------------------------------------------------------
constexpr int K1_UNROLL = 2;                        // 16-byte vectors of each input per lane per step
constexpr int K1_STAGE = 2 * K1_UNROLL * 32 * 16;   // bytes of a warp's stage (prev, cur)

// Grid origin of the MIN grid from the minimum-ratio key K0 left in the control block.
template <typename T>
__device__ __forceinline__ void anchor_min_consts(Consts<T>& c, const Ctrl* ctrl) {
  const unsigned long long key = ctrl->amin_key;
  double a = key ? key_to_ratio(key) : 0.0;
  if (a == 0.0) a = 0.0;  // a zero minimum is taken as +0
  c.a = (T)a;             // exact: the key was made from a T value
  c.af = (float)c.a;
  c.K0 = __fadd_ru(__fmul_ru(__fmul_ru(0x1p-18f, c.inv_wf), fabsf(c.af)), 0x1p-60f);
  c.C0 = __fmaf_ru(0x1p-22f, fabsf(c.af), __fadd_ru(0x1.8p-49f, 0x1p-100f));
}

// Bin of a zero change ratio (the centre of K1's shared window and of its code window).
template <typename T>
__device__ __forceinline__ int zero_change_bin(const Consts<T>& c, bool anchor_min) {
  if (!anchor_min) return 0;
  const double z = floor(-(double)c.a * (double)c.inv_w);
  return (int)fmin(fmax(z, 0.0), (double)(1 << (WIN_LOG2 + 1)));
}

// K0's per-thread part: the largest order key (= smallest binnable ratio) over elements
// j0, j0 + stride, ... < j1. Returns 0 if none is binnable.
template <typename T>
__device__ __forceinline__ unsigned long long k0_range(const T* __restrict__ prev,
                                                       const T* __restrict__ cur, int64_t j0,
                                                       int64_t j1, int64_t stride,
                                                       const Consts<T>& c) {
  unsigned long long best = 0;
  for (int64_t j = j0; j < j1; j += stride) {
    const T p = ld_stream(prev + j), x = ld_stream(cur + j);
    if (p == (T)0) continue;   // +-inf or NaN: never binnable (and a slow divide)
    const T d = t_sub(x, p);
    const T r = t_div(d, p);
    if (t_abs(r) <= c.cap) {
      const unsigned long long k = min_key(r);
      best = k > best ? k : best;
    }
  }
  return best;
}

// One warp's K0 result into the control block's key (lane 0, one atomic).
__device__ __forceinline__ void k0_publish(unsigned long long best, Ctrl* ctrl) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if (lane_id() == 0 && best) atomicMax(&ctrl->amin_key, best);
}

// Points the float32 estimate cannot decide (rare) are settled with the exact sequences 32 at a
// time, one per lane: each warp collects their element indices in its queue in shared memory
// (PQ_CAP entries) and settles a round whenever 32 are waiting, and the rest at its end, instead
// of running a round of the exact sequences, with most lanes idle, for every step that has any.
constexpr int PQ_CAP = 64;
constexpr int PQ_BYTES = PQ_CAP * 8;

struct PendQueue {
  unsigned long long* q;   // the warp's slots
  int n;                   // entries waiting (the same in every lane)
  // One round: lane l settles entry l (settle(valid, index) is called by every lane).
  template <typename Settle>
  __device__ __forceinline__ void round(int cnt, Settle& settle) {
    const int lane = (int)lane_id();
    const unsigned long long j = lane < cnt ? q[lane] : 0ull;
    const int rest = n - cnt;
    const unsigned long long t = lane < rest ? q[cnt + lane] : 0ull;
    __syncwarp();
    if (lane < rest) q[lane] = t;
    n = rest;
    __syncwarp();
    settle(lane < cnt, j);
  }
  // Queues the elements whose bit k (k < S) is set in this lane's `bits` (index(k): the
  // element's index), settling a round whenever 32 are waiting (so at most 63 ever wait).
  template <int S, typename Index, typename Settle>
  __device__ __forceinline__ void add(unsigned bits, Index index, Settle& settle) {
    if (!__any_sync(0xffffffffu, bits != 0u)) return;
    const int lane = (int)lane_id();
#pragma unroll
    for (int k = 0; k < S; ++k) {
      const bool mine = (bits >> k) & 1u;
      const unsigned bal = __ballot_sync(0xffffffffu, mine);
      if (bal == 0u) continue;
      if (mine) q[n + __popc(bal & lanemask_lt())] = index(k);
      n += __popc(bal);
      __syncwarp();
      if (n >= 32) round(32, settle);
    }
  }
  template <typename Settle>
  __device__ __forceinline__ void finish(Settle& settle) {
    if (n > 0) round(n, settle);
  }
};

// K1 over 16-byte vectors [v_lo, v_hi) of one variable (prev and cur 16-byte aligned): warp wid
// of nw takes the steps starting at v_lo + wid * 32 U, then every nw * 32 U vectors, each step
// 32 U vectors of both inputs (U = K1_UNROLL, lane l holds vectors u * 32 + l). Each warp copies
// its next step into its stage (cp.async, K1_STAGE bytes of shared memory at `stage`) before it
// classifies the current one. Codes go to codes[element], bins to the histograms of h.
template <typename T>
__device__ __forceinline__ void k1_vec_range(const HistCtx& h, const Consts<T>& c,
                                             const T* __restrict__ prev,
                                             const T* __restrict__ cur, int64_t v_lo,
                                             int64_t v_hi, int64_t wid, int64_t nw,
                                             unsigned char* stage, unsigned long long* pq,
                                             int& lmin, int& lmax) {
  using V = Vec<T>;
  using VT = typename V::type;
  const int lane = (int)lane_id();
  const VT* pv = reinterpret_cast<const VT*>(prev);
  const VT* xv = reinterpret_cast<const VT*>(cur);
  unsigned short* codes = h.codes;
  // this lane's slots of the warp's stage: [u][lane] prev vectors, then cur vectors; a lane
  // reads back only what it copied itself
  VT* sp = reinterpret_cast<VT*>(stage);
  VT* sx = sp + K1_UNROLL * 32;
  const int64_t step = nw * (32 * K1_UNROLL);
  auto stage_step = [&](int64_t b0) {
#pragma unroll
    for (int u = 0; u < K1_UNROLL; ++u) {
      const int64_t vi = b0 + u * 32 + lane;
      if (vi < v_hi) {
        cp_async16(sp + u * 32 + lane, pv + vi);
        cp_async16(sx + u * 32 + lane, xv + vi);
      }
    }
    cp_async_commit();
  };
  // the exact sequences for an element the estimate left undecided (or for nothing)
  auto settle = [&](bool valid, unsigned long long j) {
    int b = 0;
    bool binned = false, pass = false;
    if (valid) {
      binned = Classifier<T>::exact(prev[j], cur[j], c, h.cbase, b, pass) == 1;
      codes[j] = (unsigned short)bin_code(h, binned, b, pass);
    }
    hist_add(h, binned, b, lmin, lmax);
  };
  PendQueue Q{pq, 0};
  const int64_t first = v_lo + wid * (32 * K1_UNROLL);
  if (first < v_hi) stage_step(first);
  for (int64_t base = first; base < v_hi; base += step) {
    T pe[K1_UNROLL][V::N], xe[K1_UNROLL][V::N];
    bool ok[K1_UNROLL];
    cp_async_wait_all();
#pragma unroll
    for (int u = 0; u < K1_UNROLL; ++u) {
      const int64_t vi = base + u * 32 + lane;
      ok[u] = vi < v_hi;
      VT a = {}, b = {};
      if (ok[u]) { a = sp[u * 32 + lane]; b = sx[u * 32 + lane]; }
      V::get(a, pe[u]);
      V::get(b, xe[u]);
    }
    if (base + step < v_hi) stage_step(base + step);   // in flight while this step is classified
    unsigned pend = 0;   // bit u * V::N + v: element needs the exact sequences
#pragma unroll
    for (int u = 0; u < K1_UNROLL; ++u) {
      const int64_t vi = base + u * 32 + lane;
      unsigned cw[V::N];
#pragma unroll
      for (int v = 0; v < V::N; ++v) {
        int b = 0;
        bool pass = false;
        const int kind = ok[u] ? Classifier<T>::fast(pe[u][v], xe[u][v], c, h.cbase, b, pass) : 0;
        const bool binned = kind == 1;
        if (kind >= 2) pend |= 1u << (u * V::N + v);
        cw[v] = bin_code(h, binned, b, pass);
        hist_add(h, binned, b, lmin, lmax);
      }
      if (ok[u]) reinterpret_cast<typename V::codes*>(codes)[vi] = V::pack(cw);
    }
    // undecided elements (rare) wait for a round of the exact sequences
    Q.add<K1_UNROLL * V::N>(
        pend,
        [&](int k) {
          return (unsigned long long)((base + (k / V::N) * 32 + lane) * V::N + (k % V::N));
        },
        settle);
  }
  Q.finish(settle);
}

// K1 over elements [j_lo, j_hi) with scalar loads (any alignment; also the tail after the last
// whole vector): warp wid of nw takes steps of 32 U elements from j_lo + wid * 32 U.
template <typename T, int U>
__device__ __forceinline__ void k1_scalar_range(const HistCtx& h, const Consts<T>& c,
                                                const T* __restrict__ prev,
                                                const T* __restrict__ cur, int64_t j_lo,
                                                int64_t j_hi, int64_t wid, int64_t nw, int& lmin,
                                                int& lmax) {
  const int lane = (int)lane_id();
  for (int64_t base = j_lo + wid * (32 * U); base < j_hi; base += nw * (32 * U)) {
    T pe[U], xe[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = base + u * 32 + lane;
      ok[u] = j < j_hi;
      pe[u] = ok[u] ? ld_stream(prev + j) : (T)0;
      xe[u] = ok[u] ? ld_stream(cur + j) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int b = 0;
      bool pass = false;
      const bool binned = ok[u] && Classifier<T>::exact(pe[u], xe[u], c, h.cbase, b, pass) == 1;
      if (ok[u]) h.codes[base + u * 32 + lane] = (unsigned short)bin_code(h, binned, b, pass);
      hist_add(h, binned, b, lmin, lmax);
    }
  }
}

// Clears the per-tile counts of the tiles holding elements [e0, e1) of a variable (a K1 pass
// leaves them zero for K3a), all threads of the CTA; with `scan_flags` also the offset scan's
// look-back flags after them.
__device__ __forceinline__ void clear_tile_counts(unsigned long long* tstatus, const Geometry& g,
                                                  int64_t e0, int64_t e1, bool scan_flags) {
  if (e1 <= e0) return;
  const int64_t q0 = e0 / g.epb, q1 = (e1 - 1) / g.epb;
  const int64_t t0 = q0 * g.spb + (e0 - q0 * g.epb) / SUB;
  int64_t t1 = q1 * g.spb + (e1 - 1 - q1 * g.epb) / SUB + 1;
  if (scan_flags) t1 = g.nsub + g.nsub / 4096 + 2;
  for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) tstatus[i] = 0ull;
}

}  // namespace nmk
