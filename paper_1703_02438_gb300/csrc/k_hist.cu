// k_hist.cu — K0: minimum binnable ratio (ANCHOR_MIN grid origin, §IV.A computes the global
// min/max of the change ratios); K1: change ratio (Eq. 1) -> bin id -> top-k histogram
// (§IV.B.1), fused in one pass over both timesteps with 128-bit streaming loads.
//
// K1 also runs the error-bound check of §III.C for every binnable point against the centre of
// its own bin (the only centre the point can be indexed to, whichever bins are selected) and
// stores bin and outcome as a 16-bit code, so that the indexing kernel reads 2 bytes per point
// instead of both timesteps.
//
// The paper builds a local histogram per MPI rank and merges them with MPI_Allreduce (§IV.B.1).
// Here each CTA keeps a private shared-memory histogram over a 16384-bin window around the
// zero-change bin (one shared atomic per point), and each CTA merges its window into the
// global histogram once at the end.
// Bins outside the shared window go straight to the global window with one atomic.
//
// One CTA of 32 warps per SM. With 16-byte aligned inputs each warp copies its next step's prev
// and cur vectors into its stage in shared memory (cp.async) before it classifies the current
// step, so its loads stay in flight while it computes (the kernel is at its register cap: a
// second register group of inputs spilled).
#include "k1.cuh"

namespace nmk {

namespace {

// ---------------------------------------------------------------------------------------
// K0: per-element exact ratio, binnable test, max of the order key (= min ratio)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k0_anchor_min(const T* __restrict__ prev,
                                                     const T* __restrict__ cur, int64_t n,
                                                     Consts<T> c, Ctrl* ctrl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  k0_publish(k0_range<T>(prev, cur, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, n, stride, c),
             ctrl);
}

// ---------------------------------------------------------------------------------------
// K1
// ---------------------------------------------------------------------------------------
constexpr int K1_THREADS = 1024;                // one CTA per SM

template <typename T, bool VEC>
__global__ void __launch_bounds__(K1_THREADS, 1) k1_hist(const T* __restrict__ prev,
                                                      const T* __restrict__ cur, int64_t n,
                                                      Consts<T> c, int anchor_min, Ctrl* ctrl,
                                                      unsigned long long* hist,
                                                      unsigned long long* tstatus, int64_t nsub,
                                                      unsigned short* codes) {
  extern __shared__ __align__(16) unsigned int sh[];   // K1's window, then the warps' stages
  if (anchor_min) anchor_min_consts<T>(c, ctrl);
  const int c0 = zero_change_bin<T>(c, anchor_min != 0);   // centre of the shared window
  HistCtx h{sh, hist, ctrl, c0 - SH_BINS / 2, c.hbase, c0 - CODE_HALF, codes};
  k1_begin(h, tstatus, nsub);

  int lmin = 0x7FFFFFFF, lmax = (int)0x80000000;
  const int lane = (int)lane_id();
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;

  if (VEC) {
    using V = Vec<T>;
    const int64_t nvec = n / V::N;
    unsigned char* stage = reinterpret_cast<unsigned char*>(sh + SH_BINS) +
                           (threadIdx.x >> 5) * (K1_STAGE + PQ_BYTES);
    k1_vec_range<T>(h, c, prev, cur, 0, nvec, gwarp, nwarps, stage,
                    reinterpret_cast<unsigned long long*>(stage + K1_STAGE), lmin, lmax);
    // scalar tail (< V elements), one warp
    const int64_t t0 = nvec * V::N;
    if (t0 < n && gwarp == 0) {
      const int64_t j = t0 + lane;
      int b = 0;
      bool binned = false, pass = false;
      if (j < n)
        binned = Classifier<T>::exact(ld_stream(prev + j), ld_stream(cur + j), c, h.cbase, b,
                                      pass) == 1;
      if (j < n) codes[j] = (unsigned short)bin_code(h, binned, b, pass);
      hist_add(h, binned, b, lmin, lmax);
    }
  } else {
    k1_scalar_range<T, 8>(h, c, prev, cur, 0, n, gwarp, nwarps, lmin, lmax);
  }

  k1_end(h, lmin, lmax);
}

// ---------------------------------------------------------------------------------------
// Fused batch (K6): K0 and K1 of every variable of a batch in one persistent launch each.
// The work list is the concatenation of the variables' bytes (wpre); CTA b of G takes bytes
// [b WT / G, (b + 1) WT / G) and, for each variable that range covers, the elements between the
// two boundaries rounded down to a multiple of 256 (both neighbours round a shared boundary the
// same way, and a variable's last CTA ends at n). Per variable part (a segment) the CTA clears
// its shared window, runs the single-variable loop over the part with its warps, and merges the
// window into that variable's histogram; the part's per-tile counts are cleared on the way.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Consts<T> fused_consts(const FusedVar& V);
template <>
__device__ __forceinline__ Consts<double> fused_consts<double>(const FusedVar& V) { return V.cd; }
template <>
__device__ __forceinline__ Consts<float> fused_consts<float>(const FusedVar& V) { return V.cf; }

// Element boundary of work coordinate x inside variable v (see above).
__device__ __forceinline__ int64_t fused_elem(long long x, long long w_lo, long long w_hi,
                                              int64_t n, int L) {
  if (x <= w_lo) return 0;
  if (x >= w_hi) return n;
  const int64_t e = ((x - w_lo) / L) & ~(int64_t)255;
  return e < n ? e : n;
}

// Calls seg(v, e0, e1) for every variable part of this CTA's work range (uniform in the CTA).
template <typename Seg>
__device__ __forceinline__ void fused_parts(const FusedArgs& F, Seg seg) {
  const long long G = gridDim.x, b = blockIdx.x;
  const long long lo = (long long)(((__int128)F.WT * b) / G);
  const long long hi = (long long)(((__int128)F.WT * (b + 1)) / G);
  if (lo >= hi) return;
  for (int v = find_var(F.wpre, F.count, lo); v < F.count && F.wpre[v] < hi; ++v) {
    const long long w_lo = F.wpre[v], w_hi = F.wpre[v + 1];
    if (w_hi <= w_lo) continue;
    const FusedVar& V = F.vars[v];
    const int L = V.g.dtype == NUMARCK_F64 ? 8 : 4;
    const int64_t e0 = fused_elem(lo, w_lo, w_hi, V.g.n, L);
    const int64_t e1 = fused_elem(hi, w_lo, w_hi, V.g.n, L);
    if (e0 < e1) seg(v, V, e0, e1);
  }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k0_fused(FusedArgs F) {
  fused_parts(F, [&](int, const FusedVar& V, int64_t e0, int64_t e1) {
    if (V.g.anchor != NUMARCK_ANCHOR_MIN) return;
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(V.ws + V.wl.ctrl);
    if (V.g.dtype == NUMARCK_F64)
      k0_publish(k0_range<double>(static_cast<const double*>(V.prev),
                                  static_cast<const double*>(V.cur), e0 + threadIdx.x, e1,
                                  THREADS, V.cd), ctrl);
    else
      k0_publish(k0_range<float>(static_cast<const float*>(V.prev),
                                 static_cast<const float*>(V.cur), e0 + threadIdx.x, e1, THREADS,
                                 V.cf), ctrl);
  });
}

template <typename T, int THREADS>
__device__ __forceinline__ void k1_fused_part(const FusedVar& V, int64_t e0, int64_t e1,
                                              unsigned int* sh) {
  Consts<T> c = fused_consts<T>(V);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(V.ws + V.wl.ctrl);
  const bool amin = V.g.anchor == NUMARCK_ANCHOR_MIN;
  if (amin) anchor_min_consts<T>(c, ctrl);
  const int c0 = zero_change_bin<T>(c, amin);
  const int64_t n = V.g.n;
  HistCtx h{sh, reinterpret_cast<unsigned long long*>(V.ws + V.wl.hist), ctrl, c0 - SH_BINS / 2,
            c.hbase, c0 - CODE_HALF, reinterpret_cast<unsigned short*>(V.blob + V.code_off)};
  if (e0 == 0 && threadIdx.x == 0) ctrl->code_base = h.cbase;
  for (int i = threadIdx.x; i < SH_BINS; i += THREADS) sh[i] = 0u;
  clear_tile_counts(reinterpret_cast<unsigned long long*>(V.ws + V.wl.status), V.g, e0, e1,
                    e1 == n);
  __syncthreads();
  int lmin = 0x7FFFFFFF, lmax = (int)0x80000000;
  const int warp = (int)(threadIdx.x >> 5);
  const T* prev = static_cast<const T*>(V.prev);
  const T* cur = static_cast<const T*>(V.cur);
  if (V.aligned16) {
    using Vv = Vec<T>;
    const int64_t nvec = n / Vv::N;
    const int64_t v1 = e1 == n ? nvec : e1 / Vv::N;
    unsigned char* stage = reinterpret_cast<unsigned char*>(sh + SH_BINS) +
                           warp * (K1_STAGE + PQ_BYTES);
    k1_vec_range<T>(h, c, prev, cur, e0 / Vv::N, v1, warp, THREADS / 32, stage,
                    reinterpret_cast<unsigned long long*>(stage + K1_STAGE), lmin, lmax);
    if (e1 == n && nvec * Vv::N < n && warp == 0)
      k1_scalar_range<T, 1>(h, c, prev, cur, nvec * Vv::N, n, 0, 1, lmin, lmax);
  } else {
    k1_scalar_range<T, 8>(h, c, prev, cur, e0, e1, warp, THREADS / 32, lmin, lmax);
  }
  k1_end(h, lmin, lmax);
  __syncthreads();   // the window and k1_end's shared range are reused by the next part
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k1_fused(FusedArgs F) {
  extern __shared__ __align__(16) unsigned int sh[];   // the window, then the warps' stages
  fused_parts(F, [&](int, const FusedVar& V, int64_t e0, int64_t e1) {
    if (V.g.dtype == NUMARCK_F64)
      k1_fused_part<double, THREADS>(V, e0, e1, sh);
    else
      k1_fused_part<float, THREADS>(V, e0, e1, sh);
  });
}

template <int THREADS>
cudaError_t launch_k1_fused(const FusedArgs& F, int sms, cudaStream_t s) {
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = SH_BINS * sizeof(unsigned int) + (THREADS / 32) * (K1_STAGE + PQ_BYTES);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k1_fused<THREADS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1_fused<THREADS>, THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  const int blocks = sms * per_sm;
  if (F.any_min) {
    k0_fused<THREADS><<<blocks, THREADS, 0, s>>>(F);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k1_fused<THREADS><<<blocks, THREADS, smem, s>>>(F);
  return cudaGetLastError();
}

template <typename T>
const Consts<T>& consts_of(const CompressPlan& P);
template <>
const Consts<float>& consts_of<float>(const CompressPlan& P) { return P.cf; }
template <>
const Consts<double>& consts_of<double>(const CompressPlan& P) { return P.cd; }

int grid_for(int64_t work_items, int per_block_items, int max_blocks) {
  int64_t b = (work_items + per_block_items - 1) / per_block_items;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

template <typename T>
cudaError_t launch_anchor_min_t(const CompressPlan& P, cudaStream_t s) {
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl);
  const int blocks = grid_for(P.g.n, 512 * 8, P.sms * 4);
  k0_anchor_min<T><<<blocks, 512, 0, s>>>(static_cast<const T*>(P.prev),
                                          static_cast<const T*>(P.cur), P.g.n, consts_of<T>(P),
                                          ctrl);
  return cudaGetLastError();
}

template <typename T, bool VEC>
cudaError_t launch_hist_tv(const CompressPlan& P, cudaStream_t s) {
  static int occ[64] = {0};   // resident CTAs per SM, per device (0 = not configured yet)
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem =
      SH_BINS * sizeof(unsigned int) + (VEC ? (K1_THREADS / 32) * (K1_STAGE + PQ_BYTES) : 0);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k1_hist<T, VEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1_hist<T, VEC>, K1_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl);
  auto* hist = reinterpret_cast<unsigned long long*>(P.ws + P.wl.hist);
  auto* tstat = reinterpret_cast<unsigned long long*>(P.ws + P.wl.status);
  // one wave of resident CTAs; small inputs use fewer CTAs so that the shared-window set-up and
  // merge stay small next to the streaming work (at least 32 elements per thread)
  const int blocks = grid_for(P.g.n, K1_THREADS * 32, P.sms * per_sm);
  k1_hist<T, VEC><<<blocks, K1_THREADS, smem, s>>>(
      static_cast<const T*>(P.prev), static_cast<const T*>(P.cur), P.g.n, consts_of<T>(P),
      P.g.anchor == NUMARCK_ANCHOR_MIN ? 1 : 0, ctrl, hist, tstat, P.g.nsub,
      reinterpret_cast<unsigned short*>(P.blob + P.code_off));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_hist(const FusedArgs& F, int k1_threads, int sms, cudaStream_t s) {
  if (F.WT <= 0) return cudaSuccess;
  return k1_threads == 512 ? launch_k1_fused<512>(F, sms, s) : launch_k1_fused<1024>(F, sms, s);
}

cudaError_t launch_anchor_min(const CompressPlan& P, cudaStream_t s) {
  if (P.g.n == 0) return cudaSuccess;
  return P.g.dtype == NUMARCK_F64 ? launch_anchor_min_t<double>(P, s)
                                  : launch_anchor_min_t<float>(P, s);
}

cudaError_t launch_hist(const CompressPlan& P, cudaStream_t s) {
  if (P.g.dtype == NUMARCK_F64)
    return P.aligned16 ? launch_hist_tv<double, true>(P, s) : launch_hist_tv<double, false>(P, s);
  return P.aligned16 ? launch_hist_tv<float, true>(P, s) : launch_hist_tv<float, false>(P, s);
}

}  // namespace nmk
