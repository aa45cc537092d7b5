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
  const unsigned short* codes;   // K1's per-element bin codes
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

// Index of one element from its bin code (§III.C): M unless binnable, in a selected bin, and the
// error check passes. fast() never calls the exact float64 sequences: it returns UNDECIDED for
// the rare points whose bin code lies outside the code window or whose check the float32
// estimate cannot decide; exact() settles those afterwards.
constexpr unsigned UNDECIDED = 0x10000u;   // above every index (indices are < 2^16)

template <typename T>
struct Assigner;

template <>
struct Assigner<float> {
  __device__ __forceinline__ static unsigned fast(float p, float x, unsigned code, int cbase,
                                                  const Consts<float>& c, const RankView& rv,
                                                  const float* s_m, const float*,
                                                  const float* g_m, const float*, unsigned M) {
    if (code == CODE_NONE) return M;
    if (code == CODE_FAR) return UNDECIDED;
    const unsigned r = rv.lookup(cbase + (int)code);
    if (r == M) return M;
    const float m = r < (unsigned)MT_SMEM ? s_m[r] : g_m[r];
    return check_exact<float>(p, x, m, c.E_T) ? r : M;
  }
  __device__ static unsigned exact(float p, float x, unsigned code, int cbase,
                                   const Consts<float>& c, const RankView& rv, const float* g_m,
                                   const float*, unsigned M) {
    if (code == CODE_NONE) return M;
    int b = cbase + (int)code;
    if (code == CODE_FAR && !classify_exact<float>(p, x, c, b)) return M;
    const unsigned r = rv.lookup(b);
    if (r == M) return M;
    return check_exact<float>(p, x, g_m[r], c.E_T) ? r : M;
  }
};

template <>
struct Assigner<double> {
  __device__ __forceinline__ static unsigned fast(double p, double x, unsigned code, int cbase,
                                                  const Consts<double>& c, const RankView& rv,
                                                  const double* s_m, const float* s_cf,
                                                  const double* g_m, const float* g_cf,
                                                  unsigned M) {
    if (code == CODE_NONE) return M;
    if (code == CODE_FAR) return UNDECIDED;
    const unsigned r = rv.lookup(cbase + (int)code);
    if (r == M) return M;
    const float cf = r < (unsigned)MT_SMEM ? s_cf[r] : g_cf[r];
    const int d = check_f64_fast(p, x, cf, c);
    return d == 1 ? r : (d == 0 ? M : UNDECIDED);
  }
  __device__ static unsigned exact(double p, double x, unsigned code, int cbase,
                                   const Consts<double>& c, const RankView& rv, const double* g_m,
                                   const float* g_cf, unsigned M) {
    if (code == CODE_NONE) return M;
    int b = cbase + (int)code;
    if (code == CODE_FAR && !classify_f64(p, x, c, b)) return M;
    const unsigned r = rv.lookup(b);
    if (r == M) return M;
    return check_f64(p, x, g_m[r], g_cf[r], c) ? r : M;
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


constexpr int K3_WARPS = 16;                    // warps per CTA; each warp owns whole tiles
constexpr int K3_THREADS = K3_WARPS * 32;
constexpr int K3_CHUNK = 1024;                  // elements a warp indexes before packing them
constexpr int K3_UNROLL = 4;                    // 32-element steps whose loads are in flight
constexpr int K3_WARP_SMEM = K3_CHUNK * 2;      // per-warp index buffer (bytes)
constexpr int STEPS = SUB / 32;                 // 32-element steps (= ballot words) per tile

// K3a — indexing and packing. One warp processes one 4096-element tile at a time (tile
// gw, gw + W, ... for global warp gw of W): for each 1024-element chunk it indexes every
// element from K1's bin code (coalesced loads of code, p, x; lane l takes every 32nd element),
// keeps the chunk's indices in its shared buffer and bit-packs them into the index block. It
// records which points are incompressible as 16-bit half-ballots (half h of 32-element step s at
// u16 index 2s + h of the tile's own codes, which the tile has already consumed: 4s + 2h < cnt/8
// bytes < 2 cnt bytes), and the tile's incompressible count in the workspace. There is no
// dependency between tiles and no block-wide barrier after the table set-up.
template <typename T>
__global__ void __launch_bounds__(K3_THREADS, 2) k3_assign(AssignArgs<T> A) {
  __shared__ unsigned short s_rank[RW_BINS];
  __shared__ T s_m[MT_SMEM];
  __shared__ float s_cf[MT_SMEM];
  extern __shared__ __align__(16) unsigned short k3_idx[];   // [K3_WARPS][K3_CHUNK]

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
    c.K0 = __fadd_ru(__fmul_ru(__fmul_ru(0x1p-18f, c.inv_wf), fabsf(c.af)), 0x1p-60f);
  }
  const int any = ctrl->any;
  const int bmin = ctrl->sel_bmin, bmax = ctrl->sel_bmax, n_sel = ctrl->n_sel;
  const int cbase = ctrl->code_base;

  // shared rank window: the whole bin range if it fits, else centred on the zero-change bin
  int rwlo = bmin;
  if (any && bmax - bmin + 1 > RW_BINS) {
    const int c0 = cbase + CODE_HALF;
    rwlo = min(max(c0 - RW_BINS / 2, bmin), bmax - RW_BINS + 1);
  }
  for (int i = tid; i < RW_BINS; i += K3_THREADS) {
    const int b = rwlo + i;
    s_rank[i] = (any && b <= bmax) ? A.rank_of[b - c.hbase] : (unsigned short)M;
  }
  const int nm = min(n_sel, MT_SMEM);
  for (int r = tid; r < nm; r += K3_THREADS) {
    s_m[r] = A.mtab[r];
    s_cf[r] = A.cftab[r];
  }
  __syncthreads();   // the only block-wide barrier: tables are read-only from here on
  const RankView rv{s_rank, A.rank_of, rwlo, c.hbase};

  const int B = g.B;
  unsigned short* my_idx = k3_idx + warp * K3_CHUNK;
  const long long W = (long long)gridDim.x * K3_WARPS;
  for (long long gt = (long long)blockIdx.x * K3_WARPS + warp; gt < g.nsub; gt += W) {
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);
    const T* pt = A.prev + j0;
    const T* xt = A.cur + j0;
    const unsigned short* ct = A.codes + j0;
    unsigned short* halves = const_cast<unsigned short*>(A.codes) + j0;
    unsigned char* tile_out = A.blob + g.off_index + q * g.block_stride + t * (long long)(SUB / 8 * B);

    int count = 0;
    for (int c0 = 0; c0 < cnt; c0 += K3_CHUNK) {
      const int ccnt = min(K3_CHUNK, cnt - c0);
      unsigned my_ball = 0;   // lane l: incompressible ballot of step l of the chunk
      unsigned my_und = 0;    // lane l: undecided ballot of step l of the chunk
      for (int i0 = 0; i0 < K3_CHUNK / 32; i0 += K3_UNROLL) {
        T pv[K3_UNROLL], xv[K3_UNROLL];
        unsigned cv[K3_UNROLL];
#pragma unroll
        for (int u = 0; u < K3_UNROLL; ++u) {
          const int e = (i0 + u) * 32 + lane;
          pv[u] = (T)0;
          xv[u] = (T)0;
          cv[u] = CODE_NONE;
          if (e < ccnt) {
            cv[u] = __ldcs(ct + c0 + e);
            pv[u] = ld_stream(pt + c0 + e);
            xv[u] = ld_stream(xt + c0 + e);
          }
        }
#pragma unroll
        for (int u = 0; u < K3_UNROLL; ++u) {
          const int e = (i0 + u) * 32 + lane;
          unsigned idx = M;
          if (any) idx = Assigner<T>::fast(pv[u], xv[u], cv[u], cbase, c, rv, s_m, s_cf, A.mtab,
                                           A.cftab, M);
          const bool und = e < ccnt && idx == UNDECIDED;
          my_idx[e] = (unsigned short)(und ? 0u : idx);
          const unsigned ball = __ballot_sync(0xffffffffu, e < ccnt && idx == M);
          const unsigned uball = __ballot_sync(0xffffffffu, und);
          if (lane == i0 + u) { my_ball = ball; my_und = uball; }
          count += __popc(ball);
        }
      }
      // settle the undecided points exactly (rare): reload them, decide, patch the ballots
      unsigned pending = __ballot_sync(0xffffffffu, my_und != 0u);
      while (pending) {
        const int st = __ffs(pending) - 1;
        pending &= pending - 1;
        const unsigned u = __shfl_sync(0xffffffffu, my_und, st);
        bool mk = false;
        if ((u >> lane) & 1u) {
          const int e = st * 32 + lane;
          const unsigned idx = Assigner<T>::exact(pt[c0 + e], xt[c0 + e], ct[c0 + e], cbase, c,
                                                  rv, A.mtab, A.cftab, M);
          my_idx[e] = (unsigned short)idx;
          mk = idx == M;
        }
        const unsigned fix = __ballot_sync(0xffffffffu, mk);
        if (lane == st) my_ball |= fix;
        count += __popc(fix);
      }
      __syncwarp();
      // the chunk's ballots, as 16-bit halves over the tile's consumed codes
      {
        const int s0 = (c0 >> 5) + lane;     // step of this lane's ballot
        if (s0 * 32 < cnt) halves[2 * s0] = (unsigned short)(my_ball & 0xFFFFu);
        if (s0 * 32 + 16 < cnt) halves[2 * s0 + 1] = (unsigned short)(my_ball >> 16);
      }
      // bit-pack the chunk: index e at bits [e*B, e*B + B) of the tile, LSB first; the image
      // of the tile is padded with zero bytes to a multiple of 16. floor(v / B) for v < 2^15
      // is (v * ceil(2^20 / B)) >> 20 exactly (the error stays below 1/32 < 1 - (B-1)/B).
      const int nwords = ((((ccnt * B + 7) >> 3) + 15) >> 4) * 4;
      unsigned* out = reinterpret_cast<unsigned*>(tile_out + (long long)(c0 / 8) * B);
      const unsigned rB = ((1u << 20) + (unsigned)B - 1u) / (unsigned)B;
      for (int w = lane; w < nwords; w += 32) {
        const unsigned bit0 = (unsigned)w * 32u;
        int e = (int)(((unsigned long long)bit0 * rB) >> 20);
        const int e_end = min((int)(((unsigned long long)(bit0 + 31u) * rB) >> 20), ccnt - 1);
        unsigned acc = 0;
        for (; e <= e_end; ++e) {
          const int sh = e * B - (int)bit0;
          const unsigned xx = my_idx[e];
          acc |= sh >= 0 ? (xx << sh) : (xx >> (-sh));
        }
        out[w] = acc;
      }
      __syncwarp();
    }
    if (lane == 0) A.tstatus[gt] = (unsigned long long)count;
  }
}

// K3b — the incompressible offsets (§IV.C): exclusive prefix of the per-tile counts gives the
// sub-block table; its entries at block starts give the per-block table; the total is n_inc.
// Single pass: CTA k (taken in order from a ticket counter) scans 4096 counts with coalesced
// loads, publishes its aggregate, and finds the counts before it by a decoupled look-back over
// the aggregates of the CTAs before it (their work is tiny, so the waits are short; every wait
// is bounded and reports NUMARCK_ERR_TIMEOUT in the blob status on expiry).
constexpr int SC_THREADS = 1024;
constexpr int SC_PER = 4;
constexpr int SC_TILE = SC_THREADS * SC_PER;
constexpr unsigned long long SC_AGG = 1ull << 62, SC_INC = 2ull << 62, SC_VAL = (1ull << 62) - 1;
constexpr unsigned long long SC_LIMIT_NS = 2000000000ull;

__global__ void __launch_bounds__(SC_THREADS, 1) k3_scan(const unsigned long long* counts,
                                                        unsigned long long* flags, Ctrl* ctrl,
                                                        Geometry g, unsigned char* blob, int L) {
  __shared__ long long s_w[33];
  __shared__ long long s_P;
  __shared__ long long s_blk;
  const int tid = (int)threadIdx.x;
  if (tid == 0) s_blk = (long long)atomicAdd(&ctrl->ticket, 1u);
  __syncthreads();
  const long long blk = s_blk;
  const long long lo = blk * SC_TILE + (long long)tid * SC_PER;
  long long v[SC_PER];
  long long sum = 0;
#pragma unroll
  for (int k = 0; k < SC_PER; ++k) {
    v[k] = (lo + k < g.nsub) ? (long long)counts[lo + k] : 0;
    sum += v[k];
  }
  // block inclusive scan of the per-thread sums
  const int lane = (int)lane_id(), w = tid >> 5;
  long long inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  if (w == 0) {
    const long long x = s_w[lane];
    long long xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += u;
    }
    s_w[lane] = xi - x;
    if (lane == 31) s_w[32] = xi;
  }
  __syncthreads();
  if (tid == 0) {
    const long long agg = s_w[32];
    int* blob_status = reinterpret_cast<int*>(blob + offsetof(numarck_header, status));
    long long P = 0;
    if (blk == 0) {
      st_relaxed_u64(&flags[0], SC_INC | (unsigned long long)agg);
    } else {
      st_relaxed_u64(&flags[blk], SC_AGG | (unsigned long long)agg);
      long long j = blk - 1;
      unsigned spins = 0;
      unsigned long long t0 = 0;
      while (j >= 0) {
        const unsigned long long sv = ld_relaxed_u64(&flags[j]);
        const unsigned long long f = sv >> 62;
        if (f == 0) {
          if (++spins == 64) t0 = global_timer_ns();
          if (spins > 64) {
            __nanosleep(100);
            if ((spins & 63u) == 0 && global_timer_ns() - t0 > SC_LIMIT_NS) {
              atomicExch(blob_status, NUMARCK_ERR_TIMEOUT);
              break;
            }
          }
          continue;
        }
        P += (long long)(sv & SC_VAL);
        if (f == 2) break;
        --j;
      }
      st_relaxed_u64(&flags[blk], SC_INC | (unsigned long long)(P + agg));
    }
    s_P = P;
  }
  __syncthreads();
  long long run = s_P + s_w[w] + inc - sum;
  int64_t* sub_off = reinterpret_cast<int64_t*>(blob + g.off_sub_off);
  int64_t* inc_off = reinterpret_cast<int64_t*>(blob + g.off_inc_off);
#pragma unroll
  for (int k = 0; k < SC_PER; ++k) {
    const long long i = lo + k;
    if (i < g.nsub) {
      sub_off[i] = run;
      if (i % g.spb == 0) inc_off[i / g.spb] = run;
      if (i == g.nsub - 1) {
        const long long n_inc = run + v[k];
        inc_off[g.nblocks] = n_inc;
        numarck_header* h = reinterpret_cast<numarck_header*>(blob);
        h->n_inc = n_inc;
        h->total_bytes = g.off_exact + n_inc * (long long)L;
      }
      run += v[k];
    }
  }
}

// K3c — incompressible values (§III.C): each warp takes a tile, reads all of its half-ballots
// (before writing anything: the tile's own values may land on them) and its offset, then copies
// the cur values of its incompressible points, in element order, into the incompressible table
// (bit copies; only the sectors that hold those points are read).
template <typename T>
__global__ void __launch_bounds__(512) k3_exact(const T* __restrict__ cur,
                                                const unsigned short* codes, Geometry g,
                                                unsigned char* blob) {
  using U = typename Bits<T>::U;
  const int lane = (int)lane_id();
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  U* exact_u = reinterpret_cast<U*>(blob + g.off_exact);
  const int64_t* sub_off = reinterpret_cast<const int64_t*>(blob + g.off_sub_off);
  const U* xu = reinterpret_cast<const U*>(cur);
  for (long long gt = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gt < g.nsub;
       gt += W) {
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);
    const unsigned short* halves = codes + j0;
    // lane l holds the ballots of steps l, l+32, l+64, l+96
    unsigned mine[STEPS / 32];
#pragma unroll
    for (int k = 0; k < STEPS / 32; ++k) {
      const int st = k * 32 + lane;
      const unsigned lo = st * 32 < cnt ? halves[2 * st] : 0u;
      const unsigned hi = st * 32 + 16 < cnt ? halves[2 * st + 1] : 0u;
      mine[k] = lo | (hi << 16);
    }
    __syncwarp();
    long long run = sub_off[gt];
    // steps in groups of 8: the gathers of a group are in flight together before its stores
#pragma unroll
    for (int k = 0; k < STEPS / 32; ++k) {
#pragma unroll
      for (int s0 = 0; s0 < 32; s0 += 8) {
        unsigned ball[8];
        U val[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          ball[u] = __shfl_sync(0xffffffffu, mine[k], s0 + u);
          val[u] = 0;
          if ((ball[u] >> lane) & 1u) val[u] = xu[j0 + (long long)(k * 32 + s0 + u) * 32 + lane];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if ((ball[u] >> lane) & 1u) exact_u[run + __popc(ball[u] & lanemask_lt())] = val[u];
          run += __popc(ball[u]);
        }
      }
    }
  }
}

}  // namespace

template <typename T>
static cudaError_t launch_assign_t(const CompressPlan& P, cudaStream_t s, const Consts<T>& c) {
  if (P.g.nsub == 0) return cudaSuccess;   // n == 0: K2 already wrote every table
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
  A.codes = reinterpret_cast<const unsigned short*>(P.blob + code_offset(P.g));
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  const int dyn = K3_WARPS * K3_WARP_SMEM;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k3_assign<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         dyn);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_assign<T>, K3_THREADS, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)P.sms * per_sm;
  const long long need = (P.g.nsub + K3_WARPS - 1) / K3_WARPS;
  if (blocks > need) blocks = need;
  k3_assign<T><<<(int)blocks, K3_THREADS, dyn, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_offsets(const CompressPlan& P, cudaStream_t s) {
  if (P.g.nsub == 0) return cudaSuccess;
  const long long nblk = (P.g.nsub + SC_TILE - 1) / SC_TILE;
  auto* counts = reinterpret_cast<const unsigned long long*>(P.ws + P.wl.status);
  auto* flags = reinterpret_cast<unsigned long long*>(P.ws + P.wl.status) + P.g.nsub;
  k3_scan<<<(unsigned)nblk, SC_THREADS, 0, s>>>(counts, flags, reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl),
                                                P.g, P.blob, P.g.dtype == NUMARCK_F64 ? 8 : 4);
  return cudaGetLastError();
}

cudaError_t launch_exact(const CompressPlan& P, cudaStream_t s) {
  if (P.g.nsub == 0) return cudaSuccess;
  long long xb = (P.g.nsub + 15) / 16;
  if (xb > (long long)P.sms * 4) xb = (long long)P.sms * 4;
  const unsigned short* codes = reinterpret_cast<const unsigned short*>(P.blob + code_offset(P.g));
  if (P.g.dtype == NUMARCK_F64)
    k3_exact<double><<<(int)xb, 512, 0, s>>>(static_cast<const double*>(P.cur), codes, P.g, P.blob);
  else
    k3_exact<float><<<(int)xb, 512, 0, s>>>(static_cast<const float*>(P.cur), codes, P.g, P.blob);
  return cudaGetLastError();
}

cudaError_t launch_assign(const CompressPlan& P, cudaStream_t s) {
  return P.g.dtype == NUMARCK_F64 ? launch_assign_t<double>(P, s, P.cd)
                                  : launch_assign_t<float>(P, s, P.cf);
}

}  // namespace nmk
