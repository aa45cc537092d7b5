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

// ---------------------------------------------------------------------------------------
// K0: per-element exact ratio, binnable test, max of the order key (= min ratio)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k0_anchor_min(const T* __restrict__ prev,
                                                     const T* __restrict__ cur, int64_t n,
                                                     Consts<T> c, Ctrl* ctrl) {
  unsigned long long best = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const T p = ld_stream(prev + j), x = ld_stream(cur + j);
    const T d = t_sub(x, p);
    const T r = t_div(d, p);
    if (t_abs(r) <= c.cap) {
      const unsigned long long k = min_key(r);
      best = k > best ? k : best;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if (lane_id() == 0 && best) atomicMax(&ctrl->amin_key, best);
}

// ---------------------------------------------------------------------------------------
// K1
// ---------------------------------------------------------------------------------------
constexpr int K1_THREADS = 1024;                // one CTA per SM
constexpr int K1_UNROLL = 2;                    // 16-byte vectors of each input per lane per step
constexpr int K1_STAGE = 2 * K1_UNROLL * 32 * 16;   // bytes of a warp's stage (prev, cur)

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

template <typename T, bool VEC>
__global__ void __launch_bounds__(K1_THREADS, 1) k1_hist(const T* __restrict__ prev,
                                                      const T* __restrict__ cur, int64_t n,
                                                      Consts<T> c, int anchor_min, Ctrl* ctrl,
                                                      unsigned long long* hist,
                                                      unsigned long long* tstatus, int64_t nsub,
                                                      unsigned short* codes) {
  extern __shared__ __align__(16) unsigned int sh[];   // K1's window, then the warps' stages
  if (anchor_min) anchor_min_consts<T>(c, ctrl);
  int c0 = 0;  // bin of a zero change ratio: centre of the shared window
  if (anchor_min) {
    const double z = floor(-(double)c.a * (double)c.inv_w);
    c0 = (int)fmin(fmax(z, 0.0), (double)(1 << (WIN_LOG2 + 1)));
  }
  HistCtx h{sh, hist, ctrl, c0 - SH_BINS / 2, c.hbase, c0 - CODE_HALF, codes};
  k1_begin(h, tstatus, nsub);

  int lmin = 0x7FFFFFFF, lmax = (int)0x80000000;
  const int lane = (int)lane_id();
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;

  if (VEC) {
    using V = Vec<T>;
    using VT = typename V::type;
    const VT* pv = reinterpret_cast<const VT*>(prev);
    const VT* xv = reinterpret_cast<const VT*>(cur);
    const int64_t nvec = n / V::N;
    // this lane's slots of the warp's stage: [u][lane] prev vectors, then cur vectors; a lane
    // reads back only what it copied itself
    VT* sp = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(sh + SH_BINS) +
                                   (threadIdx.x >> 5) * K1_STAGE);
    VT* sx = sp + K1_UNROLL * 32;
    const int64_t step = nwarps * (32 * K1_UNROLL);
    auto stage = [&](int64_t b0) {
#pragma unroll
      for (int u = 0; u < K1_UNROLL; ++u) {
        const int64_t vi = b0 + u * 32 + lane;
        if (vi < nvec) {
          cp_async16(sp + u * 32 + lane, pv + vi);
          cp_async16(sx + u * 32 + lane, xv + vi);
        }
      }
      cp_async_commit();
    };
    if (gwarp * (32 * K1_UNROLL) < nvec) stage(gwarp * (32 * K1_UNROLL));
    for (int64_t base = gwarp * (32 * K1_UNROLL); base < nvec; base += step) {
      T pe[K1_UNROLL][V::N], xe[K1_UNROLL][V::N];
      bool ok[K1_UNROLL];
      cp_async_wait_all();
#pragma unroll
      for (int u = 0; u < K1_UNROLL; ++u) {
        const int64_t vi = base + u * 32 + lane;
        ok[u] = vi < nvec;
        VT a = {}, b = {};
        if (ok[u]) { a = sp[u * 32 + lane]; b = sx[u * 32 + lane]; }
        V::get(a, pe[u]);
        V::get(b, xe[u]);
      }
      if (base + step < nvec) stage(base + step);   // in flight while this step is classified
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
      // settle undecided elements (rare) with the exact sequences, one per lane per round
      while (__any_sync(0xffffffffu, pend != 0u)) {
        int b = 0;
        bool binned = false, pass = false;
        if (pend) {
          const int k = __ffs(pend) - 1;
          pend &= pend - 1;
          const int u = k / V::N, v = k % V::N;
          const int64_t j = (base + u * 32 + lane) * V::N + v;   // reloaded: keeps pe, xe short-lived
          binned = Classifier<T>::exact(prev[j], cur[j], c, h.cbase, b, pass) == 1;
          codes[j] = (unsigned short)bin_code(h, binned, b, pass);
        }
        hist_add(h, binned, b, lmin, lmax);
      }
    }
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
    constexpr int U = 8;
    for (int64_t base = gwarp * (32 * U); base < n; base += nwarps * (32 * U)) {
      T pe[U], xe[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = base + u * 32 + lane;
        ok[u] = j < n;
        pe[u] = ok[u] ? ld_stream(prev + j) : (T)0;
        xe[u] = ok[u] ? ld_stream(cur + j) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int b = 0;
        bool pass = false;
        const bool binned = ok[u] && Classifier<T>::exact(pe[u], xe[u], c, h.cbase, b, pass) == 1;
        if (ok[u]) codes[base + u * 32 + lane] = (unsigned short)bin_code(h, binned, b, pass);
        hist_add(h, binned, b, lmin, lmax);
      }
    }
  }

  k1_end(h, lmin, lmax);
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
  const size_t smem = SH_BINS * sizeof(unsigned int) + (VEC ? (K1_THREADS / 32) * K1_STAGE : 0);
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
