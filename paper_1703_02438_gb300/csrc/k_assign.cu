// k_assign.cu — K3: indexing (§III.C) fused with bit packing of the index table (§IV.C) and the
// order-preserving compaction of incompressible values into the incompressible table, plus the
// per-block (§IV.C) and per-sub-block offset tables.
//
// The paper assigns integer indices per rank, aligns block boundaries across ranks with MPI_Scan
// and neighbour MPI_Send/Recv, and then bit-writes each block (§IV.C). Here a tile is one
// 4096-element sub-block of an index block, so no tile straddles a block and no exchange is
// needed; the only cross-tile dependency, the number of incompressible points before a tile,
// comes from a single-pass decoupled look-back over tiles taken in order from a ticket counter
// (every wait is bounded and reports NUMARCK_ERR_TIMEOUT in the blob status on expiry).
#include <cstddef>

#include "launch.h"

namespace nmk {

namespace {

template <typename T>
struct AssignArgs {
  const T* prev;
  const T* cur;
  Consts<T> c;
  Geometry g;
  Ctrl* ctrl;
  const unsigned short* rank_of;
  const T* mtab;
  const float* cftab;
  unsigned long long* tstatus;
  unsigned char* blob;
};

struct RankView {
  const unsigned short* s;
  const unsigned short* gl;
  int lo;
  int hbase;
  __device__ __forceinline__ unsigned lookup(int b) const {
    const int i = b - lo;
    if ((unsigned)i < (unsigned)RW_BINS) return s[i];
    return gl[b - hbase];
  }
};

template <typename T>
struct Assigner;

template <>
struct Assigner<float> {
  __device__ __forceinline__ static unsigned run(float p, float x, const Consts<float>& c,
                                                 const RankView& rv, const float* s_m,
                                                 const float*, const float* g_m, const float*,
                                                 unsigned M) {
    int b = 0;
    if (!classify_exact<float>(p, x, c, b)) return M;
    const unsigned r = rv.lookup(b);
    if (r == M) return M;
    const float m = r < (unsigned)MT_SMEM ? s_m[r] : g_m[r];
    return check_exact<float>(p, x, m, c.E_T) ? r : M;
  }
};

template <>
struct Assigner<double> {
  __device__ __forceinline__ static unsigned run(double p, double x, const Consts<double>& c,
                                                 const RankView& rv, const double* s_m,
                                                 const float* s_cf, const double* g_m,
                                                 const float* g_cf, unsigned M) {
    int b = 0;
    Est est;
    if (!classify_f64(p, x, c, b, est)) return M;
    const unsigned r = rv.lookup(b);
    if (r == M) return M;
    const bool sm = r < (unsigned)MT_SMEM;
    const double m = sm ? s_m[r] : g_m[r];
    const float cf = sm ? s_cf[r] : g_cf[r];
    return check_f64(p, x, m, cf, c, est) ? r : M;
  }
};

template <typename T>
struct Bits;
template <>
struct Bits<float> {
  using U = unsigned int;
  __device__ __forceinline__ static U of(float v) { return __float_as_uint(v); }
};
template <>
struct Bits<double> {
  using U = unsigned long long;
  __device__ __forceinline__ static U of(double v) {
    return (unsigned long long)__double_as_longlong(v);
  }
};

constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_INC = 2ull << 62;
constexpr unsigned long long VAL_MASK = (1ull << 62) - 1;
constexpr unsigned long long LOOKBACK_LIMIT_NS = 2000000000ull;   // 2 s

// Decoupled look-back (one thread): publish this tile's count, sum predecessors until one
// with an inclusive prefix is found, publish the inclusive prefix. Returns the exclusive one.
__device__ long long lookback(unsigned long long* st, long long g, long long count,
                              int* blob_status) {
  if (g == 0) {
    st_relaxed_u64(&st[0], FLAG_INC | (unsigned long long)count);
    return 0;
  }
  st_relaxed_u64(&st[g], FLAG_AGG | (unsigned long long)count);
  long long P = 0;
  long long j = g - 1;
  unsigned long long t0 = 0;
  unsigned spins = 0;
  while (j >= 0) {
    const unsigned long long s = ld_relaxed_u64(&st[j]);
    const unsigned long long f = s >> 62;
    if (f == 0) {
      ++spins;
      if (spins == 32) t0 = global_timer_ns();
      if (spins > 32) {
        __nanosleep(64);
        if ((spins & 255u) == 0 && global_timer_ns() - t0 > LOOKBACK_LIMIT_NS) {
          atomicExch(blob_status, NUMARCK_ERR_TIMEOUT);
          break;
        }
      }
      continue;
    }
    P += (long long)(s & VAL_MASK);
    if (f == 2) break;
    --j;
  }
  st_relaxed_u64(&st[g], FLAG_INC | (unsigned long long)(P + count));
  return P;
}

template <typename T>
__global__ void __launch_bounds__(TILE_THREADS, 2) k3_assign(AssignArgs<T> A) {
  __shared__ unsigned short s_idx[SUB];
  __shared__ unsigned short s_rank[RW_BINS];
  __shared__ T s_m[MT_SMEM];
  __shared__ float s_cf[MT_SMEM];
  __shared__ int s_chunk[NCHUNK];
  __shared__ long long s_tile;
  __shared__ long long s_P;
  __shared__ int s_total;

  const Geometry& g = A.g;
  Ctrl* ctrl = A.ctrl;
  const int tid = (int)threadIdx.x;
  const int lane = (int)lane_id();
  const int warp = tid >> 5;
  const unsigned M = (unsigned)g.M;
  Consts<T> c = A.c;
  if (g.anchor == NUMARCK_ANCHOR_MIN) {
    c.a = (T)ctrl->a;
    c.af = (float)c.a;
    c.K0 = __fadd_ru(__fmul_ru(__fmul_ru(0x1p-22f, c.inv_wf), fabsf(c.af)), 0x1p-100f);
  }
  const int any = ctrl->any;
  const int bmin = ctrl->sel_bmin, bmax = ctrl->sel_bmax, n_sel = ctrl->n_sel;

  // shared rank window: the whole bin range if it fits, else centred on the zero-change bin
  int rwlo = bmin;
  if (any && bmax - bmin + 1 > RW_BINS) {
    int c0 = 0;
    if (g.anchor == NUMARCK_ANCHOR_MIN)
      c0 = (int)fmin(fmax(floor(-(double)c.a * (double)c.inv_w), 0.0), (double)(1 << 22));
    rwlo = min(max(c0 - RW_BINS / 2, bmin), bmax - RW_BINS + 1);
  }
  for (int i = tid; i < RW_BINS; i += TILE_THREADS) {
    const int b = rwlo + i;
    s_rank[i] = (any && b <= bmax) ? A.rank_of[b - c.hbase] : (unsigned short)M;
  }
  const int nm = min(n_sel, MT_SMEM);
  for (int r = tid; r < nm; r += TILE_THREADS) {
    s_m[r] = A.mtab[r];
    s_cf[r] = A.cftab[r];
  }
  const RankView rv{s_rank, A.rank_of, rwlo, c.hbase};

  int* blob_status = reinterpret_cast<int*>(A.blob + offsetof(numarck_header, status));
  T* exact = reinterpret_cast<T*>(A.blob + g.off_exact);
  using U = typename Bits<T>::U;
  U* exact_u = reinterpret_cast<U*>(exact);
  int64_t* sub_off = reinterpret_cast<int64_t*>(A.blob + g.off_sub_off);
  int64_t* inc_off = reinterpret_cast<int64_t*>(A.blob + g.off_inc_off);
  const int B = g.B;
  const int tile_bytes = SUB / 8 * B;

  for (;;) {
    if (tid == 0) s_tile = (long long)atomicAdd(&ctrl->ticket, 1u);
    __syncthreads();
    const long long gt = s_tile;
    if (gt >= g.nsub) break;
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);

    T pv[EPT], xv[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = k * TILE_THREADS + tid;
      pv[k] = (T)0;
      xv[k] = (T)0;
      if (e < cnt) {
        pv[k] = ld_stream(A.prev + j0 + e);
        xv[k] = ld_stream(A.cur + j0 + e);
      }
    }
    unsigned ball[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = k * TILE_THREADS + tid;
      unsigned idx = 0;
      if (e < cnt)
        idx = any ? Assigner<T>::run(pv[k], xv[k], c, rv, s_m, s_cf, A.mtab, A.cftab, M) : M;
      s_idx[e] = (unsigned short)idx;
      ball[k] = __ballot_sync(0xffffffffu, e < cnt && idx == M);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) s_chunk[k * (TILE_THREADS / 32) + warp] = __popc(ball[k]);
    }
    __syncthreads();
    if (warp == 0) {
      int v[NCHUNK / 32];
      int sum = 0;
#pragma unroll
      for (int i = 0; i < NCHUNK / 32; ++i) { v[i] = s_chunk[lane * (NCHUNK / 32) + i]; sum += v[i]; }
      const int incl = warp_incl_scan(sum);
      int ex = incl - sum;
#pragma unroll
      for (int i = 0; i < NCHUNK / 32; ++i) { s_chunk[lane * (NCHUNK / 32) + i] = ex; ex += v[i]; }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) {
        s_total = total;
        s_P = lookback(A.tstatus, gt, total, blob_status);
      }
    }
    __syncthreads();
    const long long P = s_P;

    // incompressible values, in element order (bit copies)
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if ((ball[k] >> lane) & 1u) {
        const long long pos = P + s_chunk[k * (TILE_THREADS / 32) + warp] +
                              __popc(ball[k] & lanemask_lt());
        exact_u[pos] = Bits<T>::of(xv[k]);
      }
    }

    // bit-pack the tile: index e occupies bits [e*B, e*B + B), least significant bit first
    {
      const int nbytes = (cnt * B + 7) >> 3;
      const int nv16 = (nbytes + 15) >> 4;
      uint4* out = reinterpret_cast<uint4*>(A.blob + g.off_index + q * g.block_stride +
                                            t * (long long)tile_bytes);
      for (int v = tid; v < nv16; v += TILE_THREADS) {
        unsigned w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int bit0 = (v * 4 + h) * 32;
          int e = bit0 / B;
          const int e_end = min((bit0 + 31) / B, SUB - 1);
          unsigned long long acc = 0;
          for (; e <= e_end; ++e) {
            const int sh = e * B - bit0;
            const unsigned long long x = s_idx[e];
            acc |= sh >= 0 ? (x << sh) : (x >> (-sh));
          }
          w[h] = (unsigned)acc;
        }
        out[v] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }

    if (tid == 0) {
      sub_off[gt] = P;
      if (t == 0) inc_off[q] = P;
      if (gt == g.nsub - 1) {
        const long long n_inc = P + s_total;
        inc_off[g.nblocks] = n_inc;
        numarck_header* h = reinterpret_cast<numarck_header*>(A.blob);
        h->n_inc = n_inc;
        h->total_bytes = g.off_exact + n_inc * (long long)sizeof(T);
      }
    }
    __syncthreads();
  }
}

}  // namespace

template <typename T>
static cudaError_t launch_assign_t(const CompressPlan& P, cudaStream_t s, const Consts<T>& c) {
  AssignArgs<T> A;
  A.prev = static_cast<const T*>(P.prev);
  A.cur = static_cast<const T*>(P.cur);
  A.c = c;
  A.g = P.g;
  A.ctrl = reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl);
  A.rank_of = reinterpret_cast<const unsigned short*>(P.ws + P.wl.rank);
  A.mtab = reinterpret_cast<const T*>(P.ws + P.wl.mtab);
  A.cftab = reinterpret_cast<const float*>(P.ws + P.wl.cftab);
  A.tstatus = reinterpret_cast<unsigned long long*>(P.ws + P.wl.status);
  A.blob = P.blob;
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_assign<T>,
                                                                  TILE_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)P.sms * per_sm;
  if (blocks > P.g.nsub) blocks = P.g.nsub;
  if (blocks < 1) return cudaSuccess;   // n == 0: K2 already wrote every table
  k3_assign<T><<<(int)blocks, TILE_THREADS, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_assign(const CompressPlan& P, cudaStream_t s) {
  return P.g.dtype == NUMARCK_F64 ? launch_assign_t<double>(P, s, P.cd)
                                  : launch_assign_t<float>(P, s, P.cf);
}

}  // namespace nmk
