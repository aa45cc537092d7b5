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
template <>
struct Classifier<float> {
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
  __device__ __forceinline__ static int fast(double p, double x, const Consts<double>& c,
                                             int cbase, int& b, bool& pass) {
    return classify_check_f64_fast(p, x, c, cbase, b, pass);
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

}  // namespace nmk
