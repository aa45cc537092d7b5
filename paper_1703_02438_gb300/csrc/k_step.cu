// k_step.cu — K41: one step of the closed loop in one kernel, the decompression of a blob (K4)
// fused with the first pass of the next compression (K1) against the reconstruction it makes.
//
// In the paper's in-situ use every new timestep is compressed against the reconstruction of the
// previous one (Eq. 4 chains R_i = R_{i-1} (1 + c), §III.E), so a decompression is followed by
// a compression whose prev is that decompression's output. Run one after the other, K4 writes
// R to HBM and K1 reads it back. Here each lane classifies the four points it has just
// reconstructed (Eq. 1 ratio, §IV.B.1 bin and histogram, §III.C own-bin check, 16-bit code)
// while they are still in registers, and reads only the next timestep besides: the step moves
// (1-α)L + B/8 + αL + L (decompression) + L + 2 (classification) bytes per point instead of
// that plus another L. K4 alone waits on memory and K1 alone on ALU issue, so in one kernel the
// two halves also overlap within each SM. Every output equals that of K4 followed by K1: the
// reconstruction, the codes, the histogram and the bin range.
//
// Used for the zero-centred grid only (the paper-literal grid anchored at the minimum ratio
// needs that minimum over all of R before any bin is known).
//
// Each warp works through its sub-block in 128-point steps, and every step would otherwise wait
// for two round trips to memory: its index field, prev and cur values, then the incompressible
// values that the field selects. For B <= K41_STAGE_MAX_B the warp instead copies the next
// step's prev and cur values and its index field into a stage in shared memory (cp.async) before
// it classifies the current step, so only the second round trip is left. The stages take no
// registers (K41 is at its register cap; holding the next field in a register cost more than the
// staging saved), and one 1024-thread CTA per SM keeps 32 warps resident with a single K1 window,
// which leaves the shared memory for the stages without shrinking the L1 cache.
#include <algorithm>

#include "k1.cuh"
#include "k4.cuh"

namespace nmk {

namespace {

constexpr int K41_WARPS = 32;                    // warps per CTA (each owns a sub-block or a part)
constexpr int K41_THREADS = K41_WARPS * 32;      // one CTA per SM
constexpr int K41_STAGE_MAX_B = 10;             // index lengths whose steps are staged

// Shared memory after K1's window. With B <= K41_STAGE_MAX_B: the 2^B multipliers (room for
// TAB), then one stage per warp: a step's prev values, its cur values and its 16 B bytes of index
// field. With larger B the region holds the first DM_SMEM multipliers and no step is staged.
template <typename T>
struct Stage {
  static constexpr int L = (int)sizeof(T);
  static constexpr int FIELD = 2 * K4_SEG * L;   // byte offset of the field in a stage
  static constexpr int BYTES = FIELD + 16 * K41_STAGE_MAX_B;
  static constexpr int TAB = 1 << K41_STAGE_MAX_B;
  static constexpr int REGION = std::max(TAB * L + K41_WARPS * BYTES, DM_SMEM * L);
};



// Starts the copies of the whole step at s1 (16-byte aligned inputs and tile image tw) into the
// warp's stage wst: this lane's four prev and four cur values, and (lanes 0 .. B-1) the step's
// 16 B bytes of index field.
template <typename T, int B>
__device__ __forceinline__ void stage_step(unsigned char* wst, const T* pt, const T* xt, int s1,
                                           int lane, const unsigned* tw) {
  constexpr int L = Stage<T>::L;
  T* sp = reinterpret_cast<T*>(wst);
  T* sc = sp + K4_SEG;
  const int e = s1 + 4 * lane;
#pragma unroll
  for (int c = 0; c < 4 * L / 16; ++c) {
    cp_async16(sp + 4 * lane + c * (16 / L), pt + e + c * (16 / L));
    cp_async16(sc + 4 * lane + c * (16 / L), xt + e + c * (16 / L));
  }
  if (lane < B)
    cp_async16(wst + Stage<T>::FIELD + 16 * lane,
               reinterpret_cast<const unsigned char*>(tw) + (s1 / K4_SEG) * 16 * B + 16 * lane);
  cp_async_commit();
}

struct StepArgs {
  const void* cur;               // the next timestep, n elements of T
  Ctrl* ctrl;                    // the next compression's control block
  unsigned long long* hist;      // its global histogram window
  unsigned long long* tstatus;   // its per-tile counts and offset-scan flags
  int64_t nsub;                  // its sub-block count
  unsigned short* codes;         // its per-point codes
};

template <typename T, int B>
__device__ __forceinline__ void step_tiles(const DecodeArgs& A, const StepArgs& S,
                                           const Geometry& g, long long n_inc, const T* s_m,
                                           unsigned char* stages, unsigned long long* pq,
                                           const Consts<T>& c, const HistCtx& h, int& lmin,
                                           int& lmax) {
  using U = typename BitsOf<T>::U;
  using F = typename Field<B>::type;
  constexpr int FB = 4 * B;
  constexpr bool kStage = B <= K41_STAGE_MAX_B;
  const int lane = (int)lane_id();
  const int warp = (int)(threadIdx.x >> 5);
  unsigned char* wst = stages + warp * Stage<T>::BYTES;
  const T* sp = reinterpret_cast<const T*>(wst);
  const unsigned* sw = reinterpret_cast<const unsigned*>(wst + Stage<T>::FIELD);
  const T* centres = reinterpret_cast<const T*>(A.blob + g.off_centres);
  const int64_t* idx_off = reinterpret_cast<const int64_t*>(A.blob + g.off_idx_off);
  const int64_t* sub_off = reinterpret_cast<const int64_t*>(A.blob + g.off_sub_off);
  const U* exact_u = reinterpret_cast<const U*>(A.blob + g.off_exact);
  const unsigned char* index = A.blob + g.off_index;
  const T* prev = static_cast<const T*>(A.prev_seg);
  T* out = static_cast<T*>(A.out_seg);
  const T* cur = static_cast<const T*>(S.cur);
  const unsigned lt = lanemask_lt();
  // the exact sequences for a point the estimate left undecided: its reconstruction is read back
  // from the output (written by a lane of this warp before the point was queued)
  auto settle = [&](bool valid, unsigned long long j) {
    int b = 0;
    bool binned = false, pass = false;
    if (valid) {
      binned = Classifier<T>::exact(out[j], cur[j], c, h.cbase, b, pass) == 1;
      S.codes[j] = (unsigned short)bin_code(h, binned, b, pass);
    }
    hist_add(h, binned, b, lmin, lmax);
  };
  PendQueue Q{pq + (threadIdx.x >> 5) * PQ_CAP, 0};

  const long long W = (long long)gridDim.x * K41_WARPS;
  const int sl = A.seg_log2;                     // units: 2^sl segments per sub-block
  const int seglen = SUB >> sl;
  const long long u1 = g.nsub << sl;
  for (long long u = (long long)blockIdx.x * K41_WARPS + warp; u < u1; u += W) {
    const long long gt = u >> sl;
    const int sbeg = (int)(u & ((1 << sl) - 1)) * seglen;
    const long long q = gt / g.spb, t = gt - q * g.spb;
    const long long j0 = q * g.epb + t * SUB;
    const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
    const int cnt = (int)min((long long)SUB, bend - j0);
    const long long base = sub_off[gt];
    const long long boff = idx_off[q];
    const long long tstart = boff + t * (long long)(SUB / 8 * B);
    const int twords = 4 * ((cnt * B + 127) / 128);
    if (base < 0 || base > n_inc || (boff & 15) || boff < 0 ||
        tstart + 4LL * twords > g.index_bytes) {
      if (lane == 0) report(A, NUMARCK_ERR_CORRUPT);
      continue;
    }
    const unsigned* tw = reinterpret_cast<const unsigned*>(index + tstart);
    const int send = min(cnt, sbeg + seglen);      // this warp's points [sbeg, send) of the tile
    if (sbeg >= send) continue;
    const T* pt = prev + j0;
    T* ot = out + j0;
    const T* xt = cur + j0;
    unsigned short* ct = S.codes + j0;
    const bool vec = ((reinterpret_cast<uintptr_t>(pt) | reinterpret_cast<uintptr_t>(ot) |
                       reinterpret_cast<uintptr_t>(xt)) & 15) == 0;
    const bool cvec = (reinterpret_cast<uintptr_t>(ct) & 7) == 0;
    const bool stage_ok = kStage && vec && (reinterpret_cast<uintptr_t>(tw) & 15) == 0;
    long long run = base + (sbeg ? markers_before<B>(tw, twords, cnt, sbeg, lane) : 0u);
    bool staged = false;                         // this step's inputs are in the stage
    for (int s0 = sbeg; s0 < send; s0 += K4_SEG) {
      const int e0 = s0 + 4 * lane;
      const bool whole = s0 + K4_SEG <= cnt;     // uniform across the warp
      F field;
      T pv[4], xv[4];
      if (staged) {
        cp_async_wait_all();
        __syncwarp();                            // the field words other lanes copied
        if constexpr (kStage) field = load_field_staged<B>(sw, lane);
        lds4(sp + 4 * lane, pv);
        lds4(sp + K4_SEG + 4 * lane, xv);
      } else if (vec && whole) {
        field = load_field<B>(tw, twords, (s0 / K4_SEG) * FB, lane);
        ld4(pt + e0, pv);
        ld4(xt + e0, xv);
      } else {
        field = load_field<B>(tw, twords, (s0 / K4_SEG) * FB, lane);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          pv[k] = e0 + k < cnt ? __ldcs(pt + e0 + k) : (T)0;
          xv[k] = e0 + k < cnt ? __ldcs(xt + e0 + k) : (T)0;
        }
      }
      // decompression of the four points (as K4)
      T r[4];
      const unsigned total = decode_step<T, B>(field, pv, e0, cnt, 0, cnt, run, lt, s_m, centres,
                                               exact_u, n_inc, A, r);
      run += total;
      // the next step's inputs, in flight while this step is classified
      staged = false;
      if constexpr (kStage) {
        const int s1 = s0 + K4_SEG;
        if (stage_ok && s1 < send && s1 + K4_SEG <= cnt) {
          __syncwarp();                          // every lane has read this step's field
          stage_step<T, B>(wst, pt, xt, s1, lane, tw);
          staged = true;
        }
      }
      if (vec && whole) {
        st4(ot + e0, r);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (e0 + k < cnt) ot[e0 + k] = r[k];
      }
      // first pass of the next compression on (r, x) (as K1)
      unsigned pend = 0;
      unsigned cw[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int b = 0;
        bool pass = false;
        const int kind =
            e0 + k < cnt ? Classifier<T>::template fast<false>(r[k], xv[k], c, h.cbase, b, pass) : 0;
        const bool binned = kind == 1;
        if (kind >= 2) pend |= 1u << k;
        cw[k] = bin_code(h, binned, b, pass);
        hist_add(h, binned, b, lmin, lmax);
      }
      if (cvec && whole) {
        *reinterpret_cast<uint2*>(ct + e0) = make_uint2(cw[0] | (cw[1] << 16), cw[2] | (cw[3] << 16));
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (e0 + k < cnt) ct[e0 + k] = (unsigned short)cw[k];
      }
      // undecided points (rare) wait for a round of the exact sequences
      Q.add<4>(pend, [&](int k) { return (unsigned long long)(j0 + e0 + k); }, settle);
    }
    if (send == cnt && lane == 0) {             // this warp ends the tile: all its markers seen
      const long long next = (gt + 1 < g.nsub) ? sub_off[gt + 1] : n_inc;
      if (run != next) report(A, NUMARCK_ERR_CORRUPT);
    }
  }
  Q.finish(settle);
}

template <typename T, int B = 1>
__device__ __forceinline__ void step_dispatch(const DecodeArgs& A, const StepArgs& S,
                                              const Geometry& g, long long n_inc, const T* s_m,
                                              unsigned char* stages, unsigned long long* pq,
                                              const Consts<T>& c, const HistCtx& h, int& lmin,
                                              int& lmax) {
  if constexpr (B <= NUMARCK_MAX_B) {
    if (g.B == B)
      step_tiles<T, B>(A, S, g, n_inc, s_m, stages, pq, c, h, lmin, lmax);
    else
      step_dispatch<T, B + 1>(A, S, g, n_inc, s_m, stages, pq, c, h, lmin, lmax);
  }
}

template <typename T>
__global__ void __launch_bounds__(K41_THREADS, 1) k41_step(DecodeArgs A, StepArgs S, Consts<T> c) {
  extern __shared__ __align__(16) unsigned int sh[];             // K1's shared window, then
  unsigned char* region = reinterpret_cast<unsigned char*>(sh + SH_BINS);   // Stage's region,
                                                                   // then the warps' queues
  __shared__ __align__(16) numarck_header s_h;
  __shared__ Geometry s_g;
  __shared__ int s_rc;
  // zero-centred grid: the zero-change bin is 0, the centre of the shared window
  const HistCtx h{sh, S.hist, S.ctrl, -SH_BINS / 2, c.hbase, -CODE_HALF, S.codes};
  if (threadIdx.x < NUMARCK_HEADER_BYTES / 16)
    reinterpret_cast<uint4*>(&s_h)[threadIdx.x] = reinterpret_cast<const uint4*>(A.blob)[threadIdx.x];
  k1_begin(h, S.tstatus, S.nsub);                                // ends with a block barrier
  if (threadIdx.x == 0) {
    Geometry g{};
    int rc = check_header(s_h, &g);
    if (!rc && s_h.n != A.n_expected) rc = NUMARCK_ERR_INVALID_ARG;
    if (!rc && s_h.dtype != A.dtype) rc = NUMARCK_ERR_INVALID_ARG;
    if (rc && blockIdx.x == 0) report(A, rc);
    s_rc = rc;
    s_g = g;
  }
  __syncthreads();
  int lmin = 0x7FFFFFFF, lmax = (int)0x80000000;
  if (s_rc) {
    // no reconstruction to classify: every point of the next compression is left not binnable
    // (its blob carries the error in its header)
    unsigned short* codes = S.codes;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < A.n_expected;
         j += (long long)gridDim.x * blockDim.x)
      codes[j] = (unsigned short)CODE_NONE;
  } else {
    const Geometry g = s_g;
    const int nm = min(1 << g.B, DM_SMEM);      // within TAB when B <= K41_STAGE_MAX_B
    T* s_m = reinterpret_cast<T*>(region);
    const T* centres = reinterpret_cast<const T*>(A.blob + g.off_centres);
    for (int r = threadIdx.x; r < nm; r += K41_THREADS) s_m[r] = t_add((T)1, centres[r]);
    __syncthreads();
    step_dispatch<T>(A, S, g, s_h.n_inc, s_m, region + Stage<T>::TAB * sizeof(T),
                     reinterpret_cast<unsigned long long*>(region + Stage<T>::REGION), c, h,
                     lmin, lmax);
  }
  k1_end(h, lmin, lmax);
}

template <typename T>
cudaError_t launch_step_t(const DecodePlan& D, const CompressPlan& P, cudaStream_t s) {
  static int occ[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = SH_BINS * sizeof(unsigned int) + Stage<T>::REGION + K41_WARPS * PQ_BYTES;
  int per_sm = dev < 64 ? occ[dev] : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k41_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k41_step<T>, K41_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) occ[dev] = per_sm;
  }
  // one wave of resident CTAs, fewer when the decompressed blob has fewer tiles (its tile count
  // when its header was given on the host, else the least it can have)
  long long blocks = (long long)P.sms * per_sm;
  const long long tiles = D.ntiles_hint > 0 ? D.ntiles_hint : (D.count + SUB - 1) / SUB;
  const int sl = seg_log2_for(tiles, blocks * K41_WARPS);
  blocks = std::min(blocks, std::max(1LL, ((tiles << sl) + K41_WARPS - 1) / K41_WARPS));
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(P.ws + P.wl.ctrl);
  DecodeArgs A{D.blob, D.prev_seg, D.out_seg, D.status, 0, D.count, D.n_expected, &ctrl->error,
               P.g.dtype, sl};
  StepArgs S{P.cur, ctrl, reinterpret_cast<unsigned long long*>(P.ws + P.wl.hist),
             reinterpret_cast<unsigned long long*>(P.ws + P.wl.status), P.g.nsub,
             reinterpret_cast<unsigned short*>(P.blob + P.code_off)};
  if constexpr (sizeof(T) == 8)
    k41_step<double><<<(int)blocks, K41_THREADS, smem, s>>>(A, S, P.cd);
  else
    k41_step<float><<<(int)blocks, K41_THREADS, smem, s>>>(A, S, P.cf);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(const DecodePlan& D, const CompressPlan& P, cudaStream_t s) {
  return P.g.dtype == NUMARCK_F64 ? launch_step_t<double>(D, P, s) : launch_step_t<float>(D, P, s);
}

}  // namespace nmk
