// k_assign.cu — K3: indexing (§III.C) and bit packing of the index table (§IV.C) from K1's
// per-point codes (K3a), the per-block and per-sub-block offset tables of the incompressible
// values (K3b), and the order-preserving copy of those values into the incompressible table (K3c).
//
// The paper assigns integer indices per rank, aligns block boundaries across ranks with MPI_Scan
// and neighbour MPI_Send/Recv, and then bit-writes each block (§IV.C). Here a tile is one
// 4096-element sub-block of an index block, so no tile straddles a block and no exchange is
// needed. The only cross-tile dependency, the number of incompressible points before a tile, is
// a prefix sum of per-tile counts (K3b: a single-pass decoupled look-back; every wait is bounded
// and reports NUMARCK_ERR_TIMEOUT in the blob status on expiry).
#include <array>
#include <cstddef>
#include <type_traits>
#include <utility>

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
  const unsigned short* codes;   // K1's per-point codes
};

// Rank of a bin from the global rank table (M if not selected; bins outside the selected range
// are M without a lookup). Used for the points outside K1's code window.
struct RankView {
  const unsigned short* gl;
  int hbase;
  int sel_lo, sel_hi;
  unsigned M;
  __device__ __forceinline__ unsigned lookup(int b) const {
    if (b < sel_lo || b > sel_hi) return M;
    return gl[b - hbase];
  }
};

// Index of a point whose code is CODE_FAR (binnable, bin outside K1's code window): classify
// it again with the exact sequences, look up its bin's rank, run the error-bound check (§III.C).
// Every other point's index follows from its code alone.
template <typename T>
struct FarAssigner;

template <>
struct FarAssigner<float> {
  __device__ __noinline__ static unsigned index(float p, float x, const Consts<float>& c,
                                                const RankView& rv,
                                   const float* g_m, const float*, unsigned M) {
    int b = 0;
    if (!classify_exact<float>(p, x, c, b)) return M;
    const unsigned r = rv.lookup(b);
    if (r == M) return M;
    return check_exact<float>(p, x, g_m[r], c.E_T) ? r : M;
  }
};

template <>
struct FarAssigner<double> {
  __device__ __noinline__ static unsigned index(double p, double x, const Consts<double>& c,
                                   const RankView& rv, const double* g_m, const float* g_cf,
                                   unsigned M) {
    int b = 0;
    if (!classify_f64(p, x, c, b)) return M;
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


constexpr int K3_WARPS = 32;                    // warps per CTA; each warp owns whole tiles
constexpr int K3_THREADS = K3_WARPS * 32;
constexpr int K3_SEG = 128;                     // K3f's warp step: 4 consecutive points per lane
constexpr int STEPS = SUB / 32;                 // 32-element ballot words per tile
constexpr int K3_SMEM = 65536 * 2;              // index of every 16-bit code (bytes)
// K3a's per-warp stage: one step's code vectors (32 lanes x up to 4, and lane 31's extra one)
constexpr int K3A_STAGE_U4 = 32 * 4 + 1;
constexpr int K3A_SMEM = K3_SMEM + K3_WARPS * K3A_STAGE_U4 * 16;

// K3a — indexing and packing, from K1's codes alone. One warp processes one 4096-element tile at
// a time (tile gw, gw + W, ... for global warp gw of W): index = rank of the code's bin if the
// code says the point passed the check of §III.C and the bin is selected, else the marker M
// (points with CODE_FAR are settled from prev and cur by K3f). Lane l of a step holds EL
// consecutive points (k3a_tiles), so its indices fill whole words of the step's image and its
// incompressible flags whole 16-bit half-ballot words (LSB-first order of §IV.C, zero padding to
// 16 bytes). The flags of each 16-point group go over the tile's own, already consumed codes
// (group h at u16 h of the tile's code area: h < 16 h + 16), and the tile's count of
// incompressible points to the workspace. Tiles do not depend on each other and there is no
// block-wide barrier after the rank table set-up. B is a template parameter so that the
// packing is resolved at compile time.
template <int B>
struct Field {
  using type = typename std::conditional<(4 * B <= 32), unsigned, unsigned long long>::type;
};

constexpr unsigned long long K3_FAR_FLAG = 1ull << 63;   // tile count word: far points pending

// Output of one 128-element step whose lane l holds the indices of elements e0 = sb0 + 4l ..
// e0 + 3 of the tile: incompressible flags as half-ballots, the packed B-bit fields, and the
// step's incompressible count added to `count` (group leaders only).
template <int B>
__device__ __forceinline__ void step_out(const unsigned (&idx)[4], int sb0, int cnt, int lane,
                                         unsigned short* halves, unsigned* tw, int twords,
                                         int& count) {
  using F = typename Field<B>::type;
  constexpr int FB = 4 * B;
  constexpr unsigned M = (1u << B) - 1u;
  const int e0 = sb0 + lane * 4;
  unsigned nib = 0;
  F field = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    nib |= idx[k] == M ? (1u << k) : 0u;
    field |= (F)idx[k] << (k * B);
  }
  if (sb0 + K3_SEG > cnt) {                      // last, partial step: drop points past cnt
    const int nv = min(max(cnt - e0, 0), 4);
    nib &= (1u << nv) - 1u;
    field &= nv == 4 ? ~(F)0 : (((F)1 << (nv * B)) - 1);
  }
  // incompressible flags of the step's four 32-element groups (8 lanes each)
  unsigned sb = nib << (4 * (lane & 7));
  sb |= __shfl_xor_sync(0xffffffffu, sb, 1);
  sb |= __shfl_xor_sync(0xffffffffu, sb, 2);
  sb |= __shfl_xor_sync(0xffffffffu, sb, 4);
  if ((lane & 7) == 0) {
    const int st = (sb0 >> 5) + (lane >> 3);
    if (st * 32 < cnt) halves[2 * st] = (unsigned short)(sb & 0xFFFFu);
    if (st * 32 + 16 < cnt) halves[2 * st + 1] = (unsigned short)(sb >> 16);
    count += __popc(sb);
  }
  const int wbase = (sb0 / K3_SEG) * FB;         // first word of the step in the tile image
  if constexpr (FB == 32) {
    if (wbase + lane < twords) tw[wbase + lane] = (unsigned)field;
  } else if constexpr (FB == 64) {
    const int w = wbase + 2 * lane;              // twords is even: both words or neither
    if (w < twords)
      *reinterpret_cast<uint2*>(tw + w) = make_uint2((unsigned)field, (unsigned)(field >> 32));
  } else {
    // word w of the step image takes the fields of lanes l0 .. l0 + KMAX - 1
    constexpr int KMAX = 31 / FB + 2;
    constexpr int RW = (FB + 31) / 32;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int w = lane + 32 * r;
      const int bit = w * 32;
      const int l0 = bit / FB;
      unsigned acc = 0;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int l = l0 + k;
        const F f = __shfl_sync(0xffffffffu, field, l & 31);
        const int sh = l * FB - bit;             // start of lane l's field relative to the word
        if (l < 32 && sh < 32) acc |= sh >= 0 ? (unsigned)(f << sh) : (unsigned)(f >> -sh);
      }
      if (w < FB && wbase + w < twords) tw[wbase + w] = acc;
    }
  }
}

// Geometry of tile gt: first element, element count, packed image and code area.
struct TileRef {
  long long j0;
  int cnt, twords;
  unsigned* tw;
  unsigned short* halves;
};
template <int B>
__device__ __forceinline__ TileRef tile_ref(const Geometry& g, long long gt, unsigned char* blob,
                                            const unsigned short* codes) {
  TileRef r;
  const long long q = gt / g.spb, t = gt - q * g.spb;
  r.j0 = q * g.epb + t * SUB;
  const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
  r.cnt = (int)min((long long)SUB, bend - r.j0);
  r.tw = reinterpret_cast<unsigned*>(blob + g.off_index + q * g.block_stride +
                                     t * (long long)(SUB / 8 * B));
  r.twords = 4 * ((r.cnt * B + 127) / 128);      // words of the 16-byte padded image
  r.halves = const_cast<unsigned short*>(codes) + r.j0;
  return r;
}

template <typename T>
__device__ __forceinline__ void anchor_consts(Consts<T>& c, const Geometry& g, const Ctrl* ctrl) {
  if (g.anchor == NUMARCK_ANCHOR_MIN) {
    c.a = (T)ctrl->a;
    c.af = (float)c.a;
    c.K0 = __fadd_ru(__fmul_ru(__fmul_ru(0x1p-18f, c.inv_wf), fabsf(c.af)), 0x1p-60f);
  }
}


// Codes e0 .. e0+2NW-1 of a tile (tile-relative) as NW words of two codes (the lower first),
// for a lane whose points all lie in the tile. The tile's codes start `sh` codes into the
// 16-byte-aligned word `wb` of the codes array; win holds this lane's aligned words (codes
// wb+e0 .. wb+e0+2NW-1) followed by the next 16 bytes (the next lane's first word).
template <int NW>
__device__ __forceinline__ void shifted_codes(const unsigned (&win)[NW + 4], int sh,
                                              unsigned (&cw)[NW]) {
  const bool odd = sh & 1;
  switch (sh >> 1) {                             // uniform across the warp
#define NMK_SHIFT_CASE(Q)                                                                     \
  case Q:                                                                                     \
    _Pragma("unroll") for (int i = 0; i < NW; ++i)                                            \
      cw[i] = odd ? __funnelshift_r(win[i + Q], win[i + Q + 1], 16) : win[i + Q];              \
    break;
    NMK_SHIFT_CASE(0)
    NMK_SHIFT_CASE(1)
    NMK_SHIFT_CASE(2)
    NMK_SHIFT_CASE(3)
#undef NMK_SHIFT_CASE
  }
}

// K3a's tile loop: steps of 32 EL points in which lane l holds points EL l .. EL l + EL - 1,
// EL = 16 for even B and 32 for odd B, so that its EL B-bit indices fill EL B / 32 whole 32-bit
// words of the step's image (LSB first) and its EL incompressible flags EL / 16 half-ballot
// words: the lane stores both itself, without shuffles. Codes arrive as EL / 8 16-byte loads
// per lane (a tile that starts off a 16-byte boundary funnel-shifts each lane's words with the
// next lane's). Lanes past the tile end, or whose codes would reach past the codes array, read
// their codes one by one.
// Copies into the warp's stage (cp.async, one group) this lane's code vectors of the step at sb0
// of tile t, those that lie inside the codes array, and for lane 31 of a tile that starts off a
// 16-byte boundary the vector after them. A lane reads back only what it copied itself.
template <int B>
__device__ __forceinline__ void k3a_stage(const unsigned short* codes, const Geometry& g,
                                          const TileRef& t, int sb0, uint4* stage, int lane) {
  constexpr int EL = B % 2 == 0 ? 16 : 32, NV = EL / 8;
  const int sh = (int)(t.j0 & 7);
  const long long wb = t.j0 - sh;
  const uint4* cw4 = reinterpret_cast<const uint4*>(codes + wb);
  const int e0 = sb0 + EL * lane;
  const long long w0 = wb + e0;
#pragma unroll
  for (int v = 0; v < NV; ++v)
    if (w0 + 8 * (v + 1) <= g.n) cp_async16(stage + lane * NV + v, cw4 + (e0 >> 3) + v);
  if (lane == 31 && sh && e0 + EL <= t.cnt && w0 + EL + 8 <= g.n)
    cp_async16(stage + 32 * NV, cw4 + (e0 >> 3) + NV);
  cp_async_commit();
}

// One tile gt (one warp): its packed indices, its incompressible flags as half-ballot words into
// `halves` (u16 h: points 16 h .. 16 h + 15 of the tile; the tile's own code area, or any other
// 512-byte buffer), and the return value: the tile's incompressible count, with K3_FAR_FLAG when
// points outside the code window need K3f. With a stage (K3A_STAGE_U4 vectors of shared memory,
// holding this tile's first step on entry), each step's codes come from the stage, and the next
// step's (or the first step of tile next_gt, if >= 0) are copied in while the step is indexed.
// (The flags of a step go to the first 256 codes of the tile, already consumed: the next step's
// codes start SEGW >= 512 codes in.)
template <int B, typename T>
__device__ __forceinline__ unsigned long long k3a_tile(const AssignArgs<T>& A,
                                                       const unsigned short* s_tab, long long gt,
                                                       int lane, int any, bool far_chk,
                                                       unsigned short* halves,
                                                       uint4* stage = nullptr,
                                                       long long next_gt = -1) {
  constexpr unsigned M = (1u << B) - 1u;
  constexpr bool kSentinel = B < 16;             // see k3_assign
  constexpr int EL = B % 2 == 0 ? 16 : 32, NW = EL / 2, NV = EL / 8, WL = EL * B / 32;
  constexpr int SEGW = 32 * EL;
  const Geometry& g = A.g;
  {
    const TileRef tr = tile_ref<B>(g, gt, A.blob, A.codes);
    const int cnt = tr.cnt;
    const int sh = (int)(tr.j0 & 7);
    const long long wb = tr.j0 - sh;             // 16-byte-aligned code index at or before j0
    const unsigned short* ct = A.codes + tr.j0;
    const uint4* cw4 = reinterpret_cast<const uint4*>(A.codes + wb);
    int count = 0;
    unsigned far = 0;
    for (int sb0 = 0; sb0 < cnt; sb0 += SEGW) {
      const int e0 = sb0 + EL * lane;
      const long long w0 = wb + e0;              // this lane's first aligned code
      unsigned win[NW + 4];
      if (stage) cp_async_wait_all();            // this step's group has landed
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        uint4 a = make_uint4(0u, 0u, 0u, 0u);
        if (w0 + 8 * (v + 1) <= g.n) a = stage ? stage[lane * NV + v] : __ldcs(cw4 + (e0 >> 3) + v);
        win[4 * v] = a.x; win[4 * v + 1] = a.y; win[4 * v + 2] = a.z; win[4 * v + 3] = a.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) win[NW + i] = __shfl_down_sync(0xffffffffu, win[i], 1);
      const bool inside = e0 + EL <= cnt;
      const bool whole = w0 + EL + (sh ? 8 : 0) <= g.n;
      if (lane == 31 && sh && inside && whole) {
        const uint4 b = stage ? stage[32 * NV] : __ldcs(cw4 + (e0 >> 3) + NV);
        win[NW] = b.x; win[NW + 1] = b.y; win[NW + 2] = b.z; win[NW + 3] = b.w;
      }
      if (stage) {                               // the next step's codes, in flight meanwhile
        if (sb0 + SEGW < cnt)
          k3a_stage<B>(A.codes, g, tr, sb0 + SEGW, stage, lane);
        else if (next_gt >= 0)
          k3a_stage<B>(A.codes, g, tile_ref<B>(g, next_gt, A.blob, A.codes), 0, stage, lane);
      }
      unsigned cw[NW];
      if (inside && whole) {
        if (sh == 0) {
#pragma unroll
          for (int i = 0; i < NW; ++i) cw[i] = win[i];
        } else {
          shifted_codes<NW>(win, sh, cw);
        }
      } else {
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          const unsigned lo = e0 + 2 * i < cnt ? (unsigned)ct[e0 + 2 * i] : CODE_NONE;
          const unsigned hi = e0 + 2 * i + 1 < cnt ? (unsigned)ct[e0 + 2 * i + 1] : CODE_NONE;
          cw[i] = lo | (hi << 16);
        }
      }
      __syncwarp();                              // every lane holds its codes before any flag store
      unsigned w[WL];
#pragma unroll
      for (int i = 0; i < WL; ++i) w[i] = 0u;
      unsigned fl = 0;
      // the lane's EL points: their table entries, flags and fields (disjoint, so added)
      // (chk false: no point of the variable has CODE_FAR, so every entry read is at most M)
      auto point = [&](int k, bool in, bool chk) {
        const unsigned code = (cw[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
        const unsigned r = s_tab[code];
        unsigned idx = r;
        if (chk) {
          if constexpr (kSentinel) {
            far = max(far, r);
            idx = min(r, M);
          } else {
            far |= code == CODE_FAR ? 1u : 0u;
          }
        }
        fl |= (in && idx == M) ? (1u << k) : 0u;
        idx = in ? idx : 0u;                     // zero fields past the tile end
        const int bit = k * B;
        w[bit >> 5] += idx << (bit & 31);
        if ((bit & 31) + B > 32) w[(bit >> 5) + 1] += idx >> (32 - (bit & 31));
      };
      if (inside && !far_chk) {                  // every point of the lane lies in the tile
#pragma unroll
        for (int k = 0; k < EL; ++k) point(k, true, false);
      } else if (inside) {
#pragma unroll
        for (int k = 0; k < EL; ++k) point(k, true, true);
      } else {
#pragma unroll
        for (int k = 0; k < EL; ++k) point(k, e0 + k < cnt, true);
      }
#pragma unroll
      for (int h = 0; h < EL / 16; ++h)
        if (e0 + 16 * h < cnt) halves[(e0 >> 4) + h] = (unsigned short)(fl >> (16 * h));
      count += __popc(fl);
      const int ow = (sb0 / SEGW) * (32 * WL) + lane * WL;   // first word of the lane's fields
      if (ow < tr.twords) {
        if constexpr (WL % 4 == 0) {
#pragma unroll
          for (int i = 0; i < WL; i += 4)
            *reinterpret_cast<uint4*>(tr.tw + ow + i) = make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]);
        } else if constexpr (WL % 2 == 0) {
#pragma unroll
          for (int i = 0; i < WL; i += 2)
            if (ow + i < tr.twords) *reinterpret_cast<uint2*>(tr.tw + ow + i) = make_uint2(w[i], w[i + 1]);
        } else {
#pragma unroll
          for (int i = 0; i < WL; ++i)
            if (ow + i < tr.twords) tr.tw[ow + i] = w[i];
        }
      }
    }
    count = __reduce_add_sync(0xffffffffu, count);
    const bool fix = any && __any_sync(0xffffffffu, kSentinel ? far > M : far != 0u);
    return (unsigned long long)count | (fix ? K3_FAR_FLAG : 0ull);
  }
}

// Whether K3a must look for CODE_FAR points: unless every binnable point's bin (the range K2
// recorded) lies in K1's code window, or when nothing is binnable (K2 found none, or reported
// an error).
__device__ __forceinline__ bool far_check(const Ctrl* ctrl, int any) {
  const int cb = ctrl->code_base;
  return !any || ctrl->sel_bmin < cb || ctrl->sel_bmax - cb >= CODE_BINS;
}

template <int B, typename T>
__device__ __forceinline__ void k3a_tiles(const AssignArgs<T>& A, const unsigned short* s_tab,
                                          long long gt_begin, long long gt_end, long long W,
                                          int lane, int any, uint4* stage = nullptr) {
  const bool chk = far_check(A.ctrl, any);
  if (stage && gt_begin < gt_end)
    k3a_stage<B>(A.codes, A.g, tile_ref<B>(A.g, gt_begin, A.blob, A.codes), 0, stage, lane);
  for (long long gt = gt_begin; gt < gt_end; gt += W) {
    // the flags go over the tile's own, already consumed codes
    unsigned short* own = tile_ref<B>(A.g, gt, A.blob, A.codes).halves;
    const long long next = gt + W < gt_end ? gt + W : -1;
    const unsigned long long st = k3a_tile<B>(A, s_tab, gt, lane, any, chk, own, stage, next);
    if (lane == 0) A.tstatus[gt] = st;
  }
  if (stage) cp_async_wait_all();   // (nothing is left in flight: the last step stages nothing)
}

// K3a's table of the index of every 16-bit code, built by all threads of the CTA (ends with a
// block barrier; the table is read-only afterwards): every code is a marker (M) except the pass
// codes of selected bins, which take the bin's rank. CODE_FAR's entry: a value above M when
// B < 16 (max() over a tile finds far points, min() turns them into markers); M when B = 16,
// where far points are found by comparing codes.
template <typename T, int B>
__device__ __forceinline__ void k3a_table(const AssignArgs<T>& A, unsigned short* s_tab, int any) {
  constexpr unsigned M = (1u << B) - 1u;
  constexpr unsigned FARV = B < 16 ? 0xFFFFu : M;
  const Ctrl* ctrl = A.ctrl;
  const int tid = (int)threadIdx.x;
  const int cbase = ctrl->code_base;
  const int slo = any ? ctrl->sel_lo : 1, shi = any ? ctrl->sel_hi : 0;
  const uint4 fill = make_uint4(M | (M << 16), M | (M << 16), M | (M << 16), M | (M << 16));
  for (int i = tid; i < 65536 / 8; i += blockDim.x) reinterpret_cast<uint4*>(s_tab)[i] = fill;
  __syncthreads();
  const int blo = max(slo, cbase), bhi = min(shi, cbase + CODE_BINS - 1);
  for (int b = blo + tid; b <= bhi; b += blockDim.x)
    s_tab[((b - cbase) << 1) | 1] = A.rank_of[b - A.c.hbase];
  if (tid == 0) s_tab[CODE_FAR] = (unsigned short)FARV;
  __syncthreads();
}

template <typename T, int B>
__global__ void __launch_bounds__(K3_THREADS, 1) k3_assign(AssignArgs<T> A) {
  extern __shared__ __align__(16) unsigned short s_tab[];   // [65536]: index of each code, then
  uint4* stage = reinterpret_cast<uint4*>(s_tab + 65536) +   // the warps' stages
                 (threadIdx.x >> 5) * K3A_STAGE_U4;
  const int any = A.ctrl->any;
  k3a_table<T, B>(A, s_tab, any);   // the only block-wide barriers
  const long long W = (long long)gridDim.x * K3_WARPS;
  k3a_tiles<B>(A, s_tab, (long long)blockIdx.x * K3_WARPS + (threadIdx.x >> 5), A.g.nsub, W,
               (int)lane_id(), any, stage);
}

// K3f — tiles with points outside K1's code window (flagged by K3a; rare: a bin more than 16383
// bins from the zero-change bin). Each such tile is indexed again from prev and cur with the
// exact sequences (bin, rank, check of §III.C against the selected centre), replacing K3a's
// image, ballots and count. The tile's codes are not used (K3a has written ballots over them).
// K3f's work on one flagged tile gt (one warp): the tile's image, its half-ballots (into `halves`,
// or its code area when null) and, returned, its incompressible count.
template <typename T, int B>
__device__ __forceinline__ int k3f_tile(const AssignArgs<T>& A, const Consts<T>& c,
                                        const RankView& rv, long long gt, int lane,
                                        unsigned short* halves = nullptr) {
  constexpr unsigned M = (1u << B) - 1u;
  const TileRef tr = tile_ref<B>(A.g, gt, A.blob, A.codes);
  if (!halves) halves = tr.halves;
  int count = 0;
  for (int sb0 = 0; sb0 < tr.cnt; sb0 += K3_SEG) {
    unsigned idx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = sb0 + lane * 4 + k;
      const long long j = tr.j0 + e;
      idx[k] = e < tr.cnt ? FarAssigner<T>::index(A.prev[j], A.cur[j], c, rv, A.mtab, A.cftab, M)
                          : M;
    }
    step_out<B>(idx, sb0, tr.cnt, lane, halves, tr.tw, tr.twords, count);
  }
  count = __reduce_add_sync(0xffffffffu, count);
  return count;
}

template <typename T, int B>
__global__ void __launch_bounds__(K3_THREADS) k3_fixup(AssignArgs<T> A) {
  constexpr unsigned M = (1u << B) - 1u;
  const Geometry& g = A.g;
  const Ctrl* ctrl = A.ctrl;
  const int lane = (int)lane_id();
  Consts<T> c = A.c;
  anchor_consts<T>(c, g, ctrl);
  const RankView rv{A.rank_of, c.hbase, ctrl->sel_lo, ctrl->sel_hi, M};
  const long long W = (long long)gridDim.x * K3_WARPS;
  for (long long gt = (long long)blockIdx.x * K3_WARPS + (threadIdx.x >> 5); gt < g.nsub;
       gt += W) {
    if (!(A.tstatus[gt] & K3_FAR_FLAG)) continue;   // uniform across the warp
    const int count = k3f_tile<T, B>(A, c, rv, gt, lane);
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
static_assert(SC_TILE == SCAN_TILE, "the host plans scan blocks of SCAN_TILE counts");
constexpr unsigned long long SC_AGG = 1ull << 62, SC_INC = 2ull << 62, SC_VAL = (1ull << 62) - 1;
constexpr unsigned long long SC_LIMIT_NS = 2000000000ull;

// Block blk of the scan of one variable (all threads of the CTA; blocks of a variable must be
// started in increasing order, each only after the ones before it have been started).
__device__ __forceinline__ void k3_scan_block(const unsigned long long* counts,
                                              unsigned long long* flags, long long blk,
                                              const Geometry& g, unsigned char* blob, int L) {
  __shared__ long long s_w[33];
  __shared__ long long s_P;
  const int tid = (int)threadIdx.x;
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
      while (j >= 0) {
        unsigned long long sv = 0;
        if (!bounded_wait(&flags[j], SC_LIMIT_NS, sv,
                          [](unsigned long long x) { return (x >> 62) != 0ull; })) {
          atomicExch(blob_status, NUMARCK_ERR_TIMEOUT);
          break;
        }
        P += (long long)(sv & SC_VAL);
        if ((sv >> 62) == 2) break;
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

__global__ void __launch_bounds__(SC_THREADS, 1) k3_scan(const unsigned long long* counts,
                                                        unsigned long long* flags, Ctrl* ctrl,
                                                        Geometry g, unsigned char* blob, int L) {
  __shared__ long long s_blk;
  if (threadIdx.x == 0) s_blk = (long long)atomicAdd(&ctrl->ticket, 1u);
  __syncthreads();
  k3_scan_block(counts, flags, s_blk, g, blob, L);
}

// K3c — incompressible values (§III.C). Each warp takes a tile: it gets the tile's marker flags
// as 32-bit ballots (one per 32-element step), compacts the positions of the set bits into a
// per-warp list in shared memory (popcounts and a warp scan give each step its place), then
// copies the cur values at those positions into the incompressible table from the tile's entry
// in the sub-block offset table, 32 independent loads per instruction and coalesced stores.
//
// The ballots come from the half-ballots that K3a left in the tile's code area, except when the
// table can reach the code area (off_exact + n_inc * L > code offset, i.e. roughly more than 75%
// (f64) or 50% (f32) of the points are incompressible): then a later tile's values may overwrite
// an earlier tile's half-ballots before that tile has read them, so the flags are re-derived
// from the packed indices (marker = 2^B - 1), which lie in a region no kernel writes after K3a.
constexpr int K3X_WARPS = 8;
constexpr int K3X_THREADS = K3X_WARPS * 32;
constexpr int K3X_UNROLL = 4;
constexpr int K3X_SMEM = K3X_WARPS * SUB * 2;   // per warp: up to SUB u16 positions

// K3c's work on tile gt of one variable (one warp; `list` is the warp's SUB u16 of shared memory).
template <typename T>
__device__ __forceinline__ void k3x_tile(const T* __restrict__ cur, const unsigned short* codes,
                                         const Geometry& g, unsigned char* blob, bool from_codes,
                                         long long gt, unsigned short* list, int lane) {
  using U = typename Bits<T>::U;
  U* exact_u = reinterpret_cast<U*>(blob + g.off_exact);
  const int64_t* sub_off = reinterpret_cast<const int64_t*>(blob + g.off_sub_off);
  const U* xu = reinterpret_cast<const U*>(cur);
  const int B = g.B;
  const unsigned M = (unsigned)g.M, fmask = (1u << B) - 1u;
  {
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);
    // lane l holds the ballots of steps l, l+32, l+64, l+96 (all read before any store)
    unsigned mine[STEPS / 32];
    if (from_codes) {
      const unsigned short* halves = codes + j0;
#pragma unroll
      for (int k = 0; k < STEPS / 32; ++k) {
        const int st = k * 32 + lane;
        const unsigned lo = st * 32 < cnt ? halves[2 * st] : 0u;
        const unsigned hi = st * 32 + 16 < cnt ? halves[2 * st + 1] : 0u;
        mine[k] = lo | (hi << 16);
      }
    } else {
      const unsigned* iw = reinterpret_cast<const unsigned*>(
          blob + g.off_index + q * g.block_stride + t * (long long)(SUB / 8 * B));
      // ballots staged in the last STEPS words of the list, read back before it is filled
      unsigned* staged = reinterpret_cast<unsigned*>(list + SUB) - STEPS;
#pragma unroll 4
      for (int st = 0; st < STEPS; ++st) {
        const int e = st * 32 + lane;
        bool mk = false;
        if (e < cnt) {
          const unsigned bp = (unsigned)e * (unsigned)B;
          const unsigned w = bp >> 5, o = bp & 31u;
          unsigned long long v = iw[w];
          if (o + (unsigned)B > 32u) v |= (unsigned long long)iw[w + 1] << 32;
          mk = ((unsigned)(v >> o) & fmask) == M;
        }
        const unsigned b = __ballot_sync(0xffffffffu, mk);
        if (lane == 0) staged[st] = b;
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < STEPS / 32; ++k) mine[k] = staged[k * 32 + lane];
      __syncwarp();
    }
    // compact the marker positions of the tile, in element order
    int total = 0;
#pragma unroll
    for (int k = 0; k < STEPS / 32; ++k) {
      const int c = __popc(mine[k]);
      const int incl = warp_incl_scan(c);
      int p = total + incl - c;
      unsigned m = mine[k];
      const int e0 = (k * 32 + lane) * 32;
      while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1u;
        list[p++] = (unsigned short)(e0 + bit);
      }
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const U* src = xu + j0;
    U* dst = exact_u + sub_off[gt];
    for (int i0 = 0; i0 < total; i0 += 32 * K3X_UNROLL) {
      U v[K3X_UNROLL];
#pragma unroll
      for (int u = 0; u < K3X_UNROLL; ++u) {
        const int i = i0 + u * 32 + lane;
        v[u] = i < total ? src[list[i]] : (U)0;
      }
#pragma unroll
      for (int u = 0; u < K3X_UNROLL; ++u) {
        const int i = i0 + u * 32 + lane;
        if (i < total) dst[i] = v[u];
      }
    }
    __syncwarp();   // the list is rebuilt for the next tile
  }
}

// Whether K3c takes a variable's marker flags from the half-ballots K3a left in its code area
// (see above), decided from the variable's n_inc.
template <typename T>
__device__ __forceinline__ bool k3x_from_codes(const Geometry& g, const unsigned char* blob,
                                               long long code_off) {
  const long long n_inc = reinterpret_cast<const numarck_header*>(blob)->n_inc;
  return g.off_exact + n_inc * (long long)sizeof(T) <= code_off;
}

template <typename T>
__global__ void __launch_bounds__(K3X_THREADS) k3_exact(const T* __restrict__ cur,
                                                        const unsigned short* codes, Geometry g,
                                                        unsigned char* blob, long long code_off) {
  extern __shared__ __align__(16) unsigned short k3x_list[];
  const int lane = (int)lane_id();
  unsigned short* list = k3x_list + (threadIdx.x >> 5) * SUB;
  const long long W = (long long)gridDim.x * K3X_WARPS;
  const bool from_codes = k3x_from_codes<T>(g, blob, code_off);
  for (long long gt = (long long)blockIdx.x * K3X_WARPS + (threadIdx.x >> 5); gt < g.nsub;
       gt += W)
    k3x_tile<T>(cur, codes, g, blob, from_codes, gt, list, lane);
}

// ---------------------------------------------------------------------------------------
// Fused batch (K6): K3a + K3f, K3b and K3c of every variable of a batch, one launch each.
// The work list of K3a/K3f and K3c is the concatenation of the variables' tiles (tpre), that of
// K3b the concatenation of their scan blocks (spre).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Consts<T> fused_consts(const FusedVar& V);
template <>
__device__ __forceinline__ Consts<double> fused_consts<double>(const FusedVar& V) { return V.cd; }
template <>
__device__ __forceinline__ Consts<float> fused_consts<float>(const FusedVar& V) { return V.cf; }

template <typename T>
__device__ __forceinline__ AssignArgs<T> fused_assign_args(const FusedVar& V) {
  AssignArgs<T> A;
  A.prev = static_cast<const T*>(V.prev);
  A.cur = static_cast<const T*>(V.cur);
  A.c = fused_consts<T>(V);
  A.g = V.g;
  A.ctrl = reinterpret_cast<Ctrl*>(V.ws + V.wl.ctrl);
  A.rank_of = reinterpret_cast<const unsigned short*>(V.ws + V.wl.rank);
  A.mtab = reinterpret_cast<const T*>(V.ws + V.wl.mtab);
  A.cftab = reinterpret_cast<const float*>(V.ws + V.wl.cftab);
  A.tstatus = reinterpret_cast<unsigned long long*>(V.ws + V.wl.status);
  A.blob = V.blob;
  A.codes = reinterpret_cast<const unsigned short*>(V.blob + V.code_off);
  return A;
}

// K3a over tiles [t0, t1) of one variable by all warps of the CTA (the code table built for this
// variable first), then K3f by each warp on the tiles it flagged. A is the variable's argument
// block in shared memory (read in place: a copy in registers would not fit beside the loop).
template <typename T, int B>
__device__ __forceinline__ void k3_fused_part(const AssignArgs<T>& A, long long t0, long long t1,
                                              unsigned short* s_tab) {
  constexpr unsigned M = (1u << B) - 1u;
  const int any = A.ctrl->any;
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  k3a_table<T, B>(A, s_tab, any);
  uint4* stage = reinterpret_cast<uint4*>(s_tab + 65536) + warp * K3A_STAGE_U4;
  k3a_tiles<B>(A, s_tab, t0 + warp, t1, K3_WARPS, lane, any, stage);
  __syncwarp();      // the tile counts (and flags) lane 0 stored are visible to the warp
  if (!any) return;
  Consts<T> c = A.c;
  anchor_consts<T>(c, A.g, A.ctrl);
  const RankView rv{A.rank_of, c.hbase, A.ctrl->sel_lo, A.ctrl->sel_hi, M};
  for (long long gt = t0 + warp; gt < t1; gt += K3_WARPS) {
    if (!(A.tstatus[gt] & K3_FAR_FLAG)) continue;                          // uniform in the warp
    const int count = k3f_tile<T, B>(A, c, rv, gt, lane);
    if (lane == 0) A.tstatus[gt] = (unsigned long long)count;
  }
}

template <typename T, int B = 1>
__device__ __forceinline__ void k3_fused_dispatch(const AssignArgs<T>& A, long long t0,
                                                  long long t1, unsigned short* s_tab) {
  if constexpr (B <= NUMARCK_MAX_B) {
    if (A.g.B == B)
      k3_fused_part<T, B>(A, t0, t1, s_tab);
    else
      k3_fused_dispatch<T, B + 1>(A, t0, t1, s_tab);
  }
}

// CTA b of G takes tiles [b NT / G, (b + 1) NT / G) of the list, variable by variable.
__global__ void __launch_bounds__(K3_THREADS, 1) k3_assign_fused(FusedArgs F) {
  extern __shared__ __align__(16) unsigned short s_tab[];   // [65536]: index of each code, stages
  __shared__ AssignArgs<double> s_ad;
  __shared__ AssignArgs<float> s_af;
  const long long G = gridDim.x, b = blockIdx.x;
  const long long lo = (long long)(((__int128)F.NT * b) / G);
  const long long hi = (long long)(((__int128)F.NT * (b + 1)) / G);
  if (lo >= hi) return;
  for (int v = find_var(F.tpre, F.count, lo); v < F.count && F.tpre[v] < hi; ++v) {
    const long long base = F.tpre[v];
    const long long t0 = max(lo, base) - base, t1 = min(hi, F.tpre[v + 1]) - base;
    if (t0 >= t1) continue;
    const bool f64 = F.vars[v].g.dtype == NUMARCK_F64;
    __syncthreads();   // the previous part is done with the table and the argument block
    if (threadIdx.x == 0) {
      if (f64) s_ad = fused_assign_args<double>(F.vars[v]);
      else s_af = fused_assign_args<float>(F.vars[v]);
    }
    __syncthreads();
    if (f64)
      k3_fused_dispatch<double>(s_ad, t0, t1, s_tab);
    else
      k3_fused_dispatch<float>(s_af, t0, t1, s_tab);
  }
}

// K3b: scan block t of the list (taken in list order from the batch's ticket counter).
__global__ void __launch_bounds__(SC_THREADS, 1) k3_scan_fused(FusedArgs F) {
  __shared__ long long s_blk;
  if (threadIdx.x == 0) s_blk = (long long)atomicAdd(F.ticket, 1u);
  __syncthreads();
  const long long t = s_blk;
  const int v = find_var(F.spre, F.count, t);
  const FusedVar& V = F.vars[v];
  const unsigned long long* counts = reinterpret_cast<const unsigned long long*>(V.ws + V.wl.status);
  k3_scan_block(counts, const_cast<unsigned long long*>(counts) + V.g.nsub, t - F.spre[v], V.g,
                V.blob, V.g.dtype == NUMARCK_F64 ? 8 : 4);
}

// K3c: warps over the tiles of the list.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k3_exact_fused(FusedArgs F) {
  extern __shared__ __align__(16) unsigned short k3x_list[];
  const int lane = (int)lane_id();
  unsigned short* list = k3x_list + (threadIdx.x >> 5) * SUB;
  const long long W = (long long)gridDim.x * WARPS;
  for (long long gt = (long long)blockIdx.x * WARPS + (threadIdx.x >> 5); gt < F.NT; gt += W) {
    const int v = find_var(F.tpre, F.count, gt);
    const FusedVar& V = F.vars[v];
    const unsigned short* codes = reinterpret_cast<const unsigned short*>(V.blob + V.code_off);
    const long long t = gt - F.tpre[v];
    if (V.g.dtype == NUMARCK_F64)
      k3x_tile<double>(static_cast<const double*>(V.cur), codes, V.g, V.blob,
                       k3x_from_codes<double>(V.g, V.blob, V.code_off), t, list, lane);
    else
      k3x_tile<float>(static_cast<const float*>(V.cur), codes, V.g, V.blob,
                      k3x_from_codes<float>(V.g, V.blob, V.code_off), t, list, lane);
  }
}

template <int WARPS>
cudaError_t launch_exact_fused_w(const FusedArgs& F, int sms, cudaStream_t s) {
  static int occ[64] = {0};
  const int smem = WARPS * SUB * 2;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k3_exact_fused<WARPS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_exact_fused<WARPS>, WARPS * 32,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)sms * per_sm;
  const long long need = (F.NT + WARPS - 1) / WARPS;
  if (blocks > need) blocks = need;
  k3_exact_fused<WARPS><<<(int)blocks, WARPS * 32, smem, s>>>(F);
  return cudaGetLastError();
}

template <typename T>
using K3Fn = void (*)(AssignArgs<T>);

template <typename T, int... Bs>
constexpr std::array<K3Fn<T>, sizeof...(Bs)> k3_table(std::integer_sequence<int, Bs...>) {
  return {{&k3_assign<T, Bs + 1>...}};
}
template <typename T, int... Bs>
constexpr std::array<K3Fn<T>, sizeof...(Bs)> k3f_table(std::integer_sequence<int, Bs...>) {
  return {{&k3_fixup<T, Bs + 1>...}};
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
  A.codes = reinterpret_cast<const unsigned short*>(P.blob + P.code_off);
  static const std::array<K3Fn<T>, NUMARCK_MAX_B> table =
      k3_table<T>(std::make_integer_sequence<int, NUMARCK_MAX_B>{});
  if (P.g.B < 1 || P.g.B > NUMARCK_MAX_B) return cudaErrorInvalidValue;
  const K3Fn<T> fn = table[P.g.B - 1];
  static int occ[64][NUMARCK_MAX_B + 1] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev][P.g.B] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, K3A_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, K3_THREADS, K3A_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev][P.g.B] = per_sm;
  }
  long long blocks = (long long)P.sms * per_sm;
  const long long need = (P.g.nsub + K3_WARPS - 1) / K3_WARPS;
  if (blocks > need) blocks = need;
  fn<<<(int)blocks, K3_THREADS, K3A_SMEM, s>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // K3f: tiles with points outside the code window (usually none; the kernel only reads flags)
  static const std::array<K3Fn<T>, NUMARCK_MAX_B> fix_table =
      k3f_table<T>(std::make_integer_sequence<int, NUMARCK_MAX_B>{});
  long long fblocks = (long long)P.sms * 2;
  if (fblocks > need) fblocks = need;
  fix_table[P.g.B - 1]<<<(int)fblocks, K3_THREADS, 0, s>>>(A);
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

template <typename T>
static cudaError_t launch_exact_t(const CompressPlan& P, cudaStream_t s) {
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k3_exact<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         K3X_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_exact<T>, K3X_THREADS, K3X_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)P.sms * per_sm;
  const long long need = (P.g.nsub + K3X_WARPS - 1) / K3X_WARPS;
  if (blocks > need) blocks = need;
  const unsigned short* codes = reinterpret_cast<const unsigned short*>(P.blob + P.code_off);
  k3_exact<T><<<(int)blocks, K3X_THREADS, K3X_SMEM, s>>>(static_cast<const T*>(P.cur), codes, P.g,
                                                          P.blob, (long long)P.code_off);
  return cudaGetLastError();
}

cudaError_t launch_exact(const CompressPlan& P, cudaStream_t s) {
  if (P.g.nsub == 0) return cudaSuccess;
  return P.g.dtype == NUMARCK_F64 ? launch_exact_t<double>(P, s) : launch_exact_t<float>(P, s);
}

cudaError_t launch_assign(const CompressPlan& P, cudaStream_t s) {
  return P.g.dtype == NUMARCK_F64 ? launch_assign_t<double>(P, s, P.cd)
                                  : launch_assign_t<float>(P, s, P.cf);
}

cudaError_t launch_fused_assign(const FusedArgs& F, int sms, cudaStream_t s) {
  if (F.NT <= 0) return cudaSuccess;
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k3_assign_fused,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, K3A_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_assign_fused, K3_THREADS, K3A_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  long long blocks = (long long)sms * per_sm;
  const long long need = (F.NT + K3_WARPS - 1) / K3_WARPS;
  if (blocks > need) blocks = need;
  k3_assign_fused<<<(int)blocks, K3_THREADS, K3A_SMEM, s>>>(F);
  return cudaGetLastError();
}

cudaError_t launch_fused_offsets(const FusedArgs& F, cudaStream_t s) {
  if (F.NS <= 0) return cudaSuccess;
  k3_scan_fused<<<(unsigned)F.NS, SC_THREADS, 0, s>>>(F);
  return cudaGetLastError();
}

cudaError_t launch_fused_exact(const FusedArgs& F, int sms, cudaStream_t s) {
  if (F.NT <= 0) return cudaSuccess;
  return F.exact_warps == 4 ? launch_exact_fused_w<4>(F, sms, s) : launch_exact_fused_w<8>(F, sms, s);
}

namespace {
// One thread runs the library's bounded wait on a caller's flag (numarck_selftest_wait).
__global__ void k_wait_selftest(const unsigned long long* flag, unsigned long long limit_ns,
                                int32_t* status) {
  unsigned long long v = 0;
  const bool ok = bounded_wait(flag, limit_ns, v, [](unsigned long long x) { return x != 0ull; });
  *status = ok ? NUMARCK_OK : NUMARCK_ERR_TIMEOUT;
}
}  // namespace

cudaError_t launch_wait_selftest(const unsigned long long* flag, unsigned long long limit_ns,
                                 int32_t* status, cudaStream_t s) {
  k_wait_selftest<<<1, 1, 0, s>>>(flag, limit_ns, status);
  return cudaGetLastError();
}

}  // namespace nmk
