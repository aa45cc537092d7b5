// k_zlib.cu — lossless compression of the index table (§IV.C: "NUMARCK splits the index table
// into blocks of same size and compresses each block using the ZLIB"), as zlib streams (RFC
// 1950) of DEFLATE data (RFC 1951) that any inflater reads, and the matching GPU inflater.
//
// Stream layout of index block q (the block's ceil(count * B / 8) bytes, without the 16-byte
// padding of the raw blob):
//   0x78 0x01                                       zlib header (deflate, 32 KB window)
//   for each 4096-element sub-block t of the block:
//     one fixed-Huffman DEFLATE block (BFINAL 0) of t's bytes, then an empty stored block
//     (BFINAL 0, BTYPE 00, LEN 0, NLEN 0xFFFF) that ends t's data on a byte boundary; or, when
//     that would be larger than t's bytes, one stored block (BFINAL 0, BTYPE 00) holding them
//   0x03 0x00                                       empty fixed-Huffman block with BFINAL 1
//   Adler-32 of the block's bytes, big-endian
// Matches never reach before the start of their sub-block, so every sub-block's data can be
// inflated on its own from its byte offset: a partial decompression inflates only the
// sub-blocks it decodes (the economics of Table 7).
//
// Match finding: a run of equal B-bit indices repeats the byte pattern with period
// p = B / gcd(B, 8) bytes (1 for B = 8, 5 for B = 10, ...), so LZ77 matches are taken at
// distance p only. A warp encodes one sub-block: lane l parses the l-th 1/32 of its bytes
// greedily (a match of length >= 3 where the bytes equal those p before, else a literal;
// matches stop at the lane's chunk end), the lanes' bit counts are scanned, and each lane writes
// its codes at its bit offset. Z1 counts bits and Adler-32 partial sums, Z2 scans the sizes into
// offsets, Z3 writes the streams; Z4 inflates sub-blocks.
#include <cstring>

#include "launch.h"

namespace nmk {

namespace {

constexpr int ZW = 4;                             // warps per CTA (one sub-block each)
constexpr int ZT = ZW * 32;
// per warp: the sub-block's image (SUB/8 * B bytes) and, in Z3, its codes (every byte a 9-bit
// literal at worst, plus the block header and tail); shared memory is sized for the blob's B
__host__ __device__ constexpr int z_in_bytes(int B) { return SUB / 8 * B; }
__host__ __device__ constexpr int z_out_words(int B) { return (z_in_bytes(B) * 9 + 64 + 31) / 32 + 4; }
constexpr unsigned ADLER = 65521u;
static_assert(sizeof(numarck_zindex_header) == NUMARCK_ZINDEX_HEADER_BYTES, "container header");

// RFC 1951 §3.2.5: length codes 257..285 (base length, extra bits).
__constant__ unsigned short c_len_base[29] = {3,  4,  5,  6,  7,  8,  9,  10, 11,  13,
                                              15, 17, 19, 23, 27, 31, 35, 43, 51,  59,
                                              67, 83, 99, 115, 131, 163, 195, 227, 258};
__constant__ unsigned char c_len_extra[29] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2,
                                              2, 3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 5, 0};
// distance codes 0..29 (base, extra bits)
__constant__ unsigned short c_dist_base[30] = {1,    2,    3,    4,    5,    7,     9,    13,
                                               17,   25,   33,   49,   65,   97,    129,  193,
                                               257,  385,  513,  769,  1025, 1537,  2049, 3073,
                                               4097, 6145, 8193, 12289, 16385, 24577};
__constant__ unsigned char c_dist_extra[30] = {0, 0, 0, 0, 1, 1, 2, 2, 3,  3,  4,  4,  5,  5,  6,
                                               6, 7, 7, 8, 8, 9, 9, 10, 10, 11, 11, 12, 12, 13, 13};

__device__ __forceinline__ unsigned rev(unsigned code, int len) {
  return __brev(code) >> (32 - len);
}

// Fixed Huffman code of a literal/length symbol (RFC 1951 §3.2.6), bit-reversed for the
// LSB-first stream; *len receives its length.
__device__ __forceinline__ unsigned fixed_code(unsigned sym, int* len) {
  if (sym < 144) { *len = 8; return rev(0x30u + sym, 8); }
  if (sym < 256) { *len = 9; return rev(0x190u + (sym - 144), 9); }
  if (sym < 280) { *len = 7; return rev(sym - 256, 7); }
  *len = 8;
  return rev(0xC0u + (sym - 280), 8);
}

__device__ __forceinline__ int len_code(int len) {   // index into c_len_base
  int c = 0;
  while (c < 28 && c_len_base[c + 1] <= len) ++c;
  return c;
}
__device__ __forceinline__ int dist_code(int d) {
  int c = 0;
  while (c < 29 && c_dist_base[c + 1] <= d) ++c;
  return c;
}

// Bits of a match (length len >= 3, distance d): length code, extra bits, distance code, extra.
__device__ __forceinline__ int match_bits(int len, int d) {
  const int lc = len_code(len), dc = dist_code(d);
  int l;
  fixed_code(257 + lc, &l);
  return l + c_len_extra[lc] + 5 + c_dist_extra[dc];
}

struct BitWriter {
  unsigned* w;        // shared words (zeroed)
  int pos;            // bit position
  __device__ __forceinline__ void put(unsigned v, int n) {   // n <= 25 bits, LSB first
    if (n == 0) return;
    const int wi = pos >> 5, sh = pos & 31;
    atomicOr(&w[wi], v << sh);
    if (sh + n > 32) atomicOr(&w[wi + 1], v >> (32 - sh));
    pos += n;
  }
};

// One lane's codes, written from a register accumulator: the words that only this lane writes
// are stored whole; its first word (shared with the codes before it) and its last (shared with
// the codes after it) are or-ed in. The words must be zero beforehand.
struct LaneBits {
  unsigned* w;
  int wi;                 // word the accumulator's bit 0 belongs to
  int first;              // this lane's first word
  unsigned long long acc;
  int nacc;               // bits held in acc (including the lane's offset into its first word)
  __device__ __forceinline__ LaneBits(unsigned* w_, int bitpos)
      : w(w_), wi(bitpos >> 5), first(bitpos >> 5), acc(0ull), nacc(bitpos & 31) {}
  __device__ __forceinline__ void put(unsigned v, int n) {   // n <= 25 bits, LSB first
    if (n == 0) return;
    acc |= (unsigned long long)v << nacc;
    nacc += n;
    if (nacc >= 32) {
      if (wi == first) atomicOr(&w[wi], (unsigned)acc);
      else w[wi] = (unsigned)acc;
      ++wi;
      acc >>= 32;
      nacc -= 32;
    }
  }
  __device__ __forceinline__ void flush() {
    if (nacc > 0) atomicOr(&w[wi], (unsigned)acc);
  }
};

struct ZArgs {
  const unsigned char* blob;
  Geometry g;
  unsigned char* z;          // container
  int64_t* tile_bytes;       // per sub-block: its slot's bytes (Z1), then its offset (Z2)
  unsigned* adler_a;         // per sub-block: sum of bytes mod 65521
  unsigned* adler_w;         // per sub-block: sum of (size - j) * byte_j mod 65521
  unsigned short* lane_bits; // per sub-block and lane: bits of the lane's codes (Z1 for Z3)
  numarck_zindex_header zh;  // container header (written into the container by Z2)
};

// The sub-block's image: tile gt of the blob (bytes [0, tb)).
struct ZTile {
  const unsigned char* src;
  int tb;                    // ceil(cnt * B / 8)
  int padded;                // the raw image's bytes (a multiple of 16, zero after tb)
  bool first, last;          // first / last sub-block of its index block
  long long q, t;
};
__device__ __forceinline__ ZTile ztile(const ZArgs& A, long long gt) {
  const Geometry& g = A.g;
  ZTile z;
  z.q = gt / g.spb;
  z.t = gt - z.q * g.spb;
  const long long j0 = z.q * g.epb + z.t * SUB;
  const long long bend = min((long long)g.n, (long long)((z.q + 1) * g.epb));
  const int cnt = (int)min((long long)SUB, bend - j0);
  z.tb = (cnt * g.B + 7) / 8;
  z.padded = 16 * ((cnt * g.B + 127) / 128);
  z.src = A.blob + g.off_index + z.q * g.block_stride + z.t * (long long)(SUB / 8 * g.B);
  z.first = z.t == 0;
  z.last = j0 + cnt == bend;
  return z;
}

// Greedy parse of bytes [c0, c1) of s with matches at distance p; bits of the codes, and (when
// bw is given) the codes themselves.
template <typename Writer>
__device__ int parse_chunk(const unsigned char* s, int c0, int c1, int p, Writer* bw) {
  int bits = 0;
  int i = c0;
  while (i < c1) {
    int len = 0;
    if (i >= p) {
      while (i + len < c1 && len < 258 && s[i + len] == s[i + len - p]) ++len;
    }
    if (len >= 3) {
      const int lc = len_code(len), dc = dist_code(p);
      if (bw) {
        int l;
        const unsigned code = fixed_code(257 + lc, &l);
        bw->put(code, l);
        bw->put((unsigned)(len - c_len_base[lc]), c_len_extra[lc]);
        bw->put(rev((unsigned)dc, 5), 5);
        bw->put((unsigned)(p - c_dist_base[dc]), c_dist_extra[dc]);
      }
      bits += match_bits(len, p);
      i += len;
    } else {
      int l;
      const unsigned code = fixed_code(s[i], &l);
      if (bw) bw->put(code, l);
      bits += l;
      ++i;
    }
  }
  return bits;
}

__device__ __forceinline__ int period_of(int B) {
  int a = B, b = 8;
  while (b) { const int t = a % b; a = b; b = t; }
  return B / a;
}

// Bytes of a sub-block's DEFLATE data: fixed Huffman (3 header bits, codes, end-of-block, then
// the empty stored block: 3 bits, padding, 4 bytes) or stored (header byte, LEN, NLEN, bytes),
// whichever is smaller (stored on ties: fixed_bytes <= stored_bytes selects fixed).
__device__ __forceinline__ int fixed_bytes(int code_bits) { return (3 + code_bits + 7 + 3 + 7) / 8 + 4; }
__device__ __forceinline__ int stored_bytes(int tb) { return 1 + 4 + tb; }
// A slot adds the zlib header before the first sub-block of a block and the final block and
// Adler-32 after the last.
__device__ __forceinline__ long long slot_bytes(int data_bytes, bool first, bool last) {
  return data_bytes + (first ? 2 : 0) + (last ? 6 : 0);
}

// Z1: per sub-block, the slot size and the Adler-32 partial sums.
__global__ void __launch_bounds__(ZT) z1_size(ZArgs A) {
  extern __shared__ __align__(16) unsigned char z_smem[];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int p = period_of(A.g.B);
  unsigned char* s = z_smem + warp * z_in_bytes(A.g.B);
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.padded / 16; i += 32)
      reinterpret_cast<uint4*>(s)[i] = __ldg(reinterpret_cast<const uint4*>(z.src) + i);
    __syncwarp();
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    int bits = parse_chunk<LaneBits>(s, c0, c1, p, nullptr);
    A.lane_bits[gt * 32 + lane] = (unsigned short)bits;
    unsigned a = 0;
    unsigned long long w = 0;
    for (int i = lane; i < z.tb; i += 32) {
      a += s[i];
      w += (unsigned long long)(z.tb - i) * s[i];
    }
    bits = __reduce_add_sync(0xffffffffu, bits);
    a = __reduce_add_sync(0xffffffffu, a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) {
      A.tile_bytes[gt] = slot_bytes(min(fixed_bytes(bits), stored_bytes(z.tb)), z.first, z.last);
      A.adler_a[gt] = a % ADLER;
      A.adler_w[gt] = (unsigned)(w % ADLER);
    }
    __syncwarp();
  }
}

// Z2: exclusive scan of the slot sizes (one CTA), per-block stream offsets, container header.
__global__ void __launch_bounds__(1024) z2_scan(ZArgs A) {
  __shared__ long long s_w[33];
  __shared__ long long s_carry;
  const Geometry& g = A.g;
  const int tid = (int)threadIdx.x, lane = (int)lane_id(), w = tid >> 5;
  int64_t* zoff = reinterpret_cast<int64_t*>(A.z + A.zh.off_zoff);
  int64_t* sub_zoff = reinterpret_cast<int64_t*>(A.z + A.zh.off_sub_zoff);
  const long long data0 = A.zh.off_data;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (long long base = 0; base < g.nsub; base += 1024) {
    const long long i = base + tid;
    const long long v = i < g.nsub ? A.tile_bytes[i] : 0;
    long long inc = v;
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
    if (i < g.nsub) {
      const long long off = data0 + s_carry + s_w[w] + inc - v;   // start of this slot
      const long long q = i / g.spb, t = i - q * g.spb;
      A.tile_bytes[i] = off;
      sub_zoff[i] = off + (t == 0 ? 2 : 0);                        // the sub-block's DEFLATE data
      if (t == 0) zoff[q] = off;
    }
    __syncthreads();
    if (tid == 0) s_carry += s_w[32];
    __syncthreads();
  }
  if (tid == 0) {
    zoff[g.nblocks] = data0 + s_carry;
    const numarck_zindex_header h = A.zh;
    const uint4* src = reinterpret_cast<const uint4*>(&h);
    uint4* dst = reinterpret_cast<uint4*>(A.z);
#pragma unroll
    for (int i = 0; i < NUMARCK_ZINDEX_HEADER_BYTES / 16; ++i) dst[i] = src[i];
  }
}

// Z3: writes every slot (zlib header, the sub-block's DEFLATE data, stream trailer).
__global__ void __launch_bounds__(ZT) z3_write(ZArgs A) {
  extern __shared__ __align__(16) unsigned char z_smem[];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int p = period_of(A.g.B);
  const int inb = z_in_bytes(A.g.B), outw = z_out_words(A.g.B);
  unsigned char* s = z_smem + warp * inb;
  unsigned* o = reinterpret_cast<unsigned*>(z_smem + ZW * inb) + warp * outw;
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.padded / 16; i += 32)
      reinterpret_cast<uint4*>(s)[i] = __ldg(reinterpret_cast<const uint4*>(z.src) + i);
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    const int bits = A.lane_bits[gt * 32 + lane];    // Z1's count of this lane's code bits
    int incl = bits;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    // the words the codes (header, codes, end of block, stored-block header bits) touch start at 0
    const int used_words = (3 + total + 10 + 31) / 32 + 1;
    for (int i = lane; i < used_words; i += 32) o[i] = 0u;
    __syncwarp();
    const long long off = A.tile_bytes[gt];
    unsigned char* dst = A.z + off;
    const int k = z.first ? 2 : 0;
    if (z.first && lane == 0) { dst[0] = 0x78; dst[1] = 0x01; }
    int nb;                                // bytes of the sub-block's DEFLATE data
    if (fixed_bytes(total) > stored_bytes(z.tb)) {
      // stored block: BFINAL 0, BTYPE 00 (the rest of the header byte is padding), LEN, NLEN
      if (lane == 0) {
        dst[k] = 0x00;
        dst[k + 1] = (unsigned char)z.tb; dst[k + 2] = (unsigned char)(z.tb >> 8);
        dst[k + 3] = (unsigned char)~z.tb; dst[k + 4] = (unsigned char)(~z.tb >> 8);
      }
      for (int i = lane; i < z.tb; i += 32) dst[k + 5 + i] = s[i];
      nb = stored_bytes(z.tb);
    } else {
      LaneBits bw(o, 3 + incl - bits);
      if (lane == 0) {
        BitWriter hw{o, 0};
        hw.put(2u, 3);                       // BFINAL 0, BTYPE 01 (fixed Huffman)
      }
      parse_chunk(s, c0, c1, p, &bw);
      bw.flush();
      __syncwarp();
      int end_bits = 3 + total;
      if (lane == 0) {
        BitWriter ew{o, end_bits};
        ew.put(0u, 7);                       // end of block (symbol 256)
        ew.put(0u, 3);                       // BFINAL 0, BTYPE 00 (stored), LEN 0 follows
      }
      __syncwarp();
      end_bits += 10;
      const int cb = (end_bits + 7) / 8;     // bytes of codes, padded to a byte boundary
      const unsigned char* ob = reinterpret_cast<const unsigned char*>(o);
      for (int i = lane; i < cb; i += 32) dst[k + i] = ob[i];
      if (lane == 0) {
        unsigned char* tail = dst + k + cb;
        tail[0] = 0x00; tail[1] = 0x00; tail[2] = 0xFF; tail[3] = 0xFF;   // LEN 0, NLEN 0xFFFF
      }
      nb = cb + 4;
    }
    if (z.last) {
      // Adler-32 of the block from its sub-blocks' partial sums (the lanes share them out): with
      // N the block's bytes and `after` the bytes of the block after sub-block u,
      // a = 1 + sum_u a_u, b = N + sum_u (after_u * a_u + w_u) (mod 65521). Every sub-block
      // before the last one of a block is full (SUB/8 * B bytes).
      const long long g0 = z.q * A.g.spb;
      const long long full = SUB / 8 * A.g.B;
      unsigned long long sa = 0, sb = 0;
      for (long long u = g0 + lane; u <= gt; u += 32) {
        const long long after = u == gt ? 0 : (long long)z.tb + (gt - 1 - u) * full;
        sa += A.adler_a[u];
        sb += ((unsigned long long)(after % ADLER) * A.adler_a[u] + A.adler_w[u]) % ADLER;
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, d);
        sb += __shfl_xor_sync(0xffffffffu, sb, d);
      }
      if (lane == 0) {
        unsigned char* tail = dst + k + nb;
        tail[0] = 0x03; tail[1] = 0x00;    // empty fixed-Huffman block with BFINAL 1
        const long long N = (long long)z.tb + (gt - g0) * full;
        sb = (sb + (unsigned long long)(N % ADLER)) % ADLER;
        sa = (1 + sa) % ADLER;
        const unsigned ad = (unsigned)((sb << 16) | sa);
        tail[2] = (unsigned char)(ad >> 24); tail[3] = (unsigned char)(ad >> 16);
        tail[4] = (unsigned char)(ad >> 8);  tail[5] = (unsigned char)ad;
      }
    }
    __syncwarp();
  }
}

// Z4: inflate sub-blocks [g0, g1] back into the raw index section of a blob (the fixed-Huffman
// and stored blocks this encoder writes; anything else is reported as NUMARCK_ERR_CORRUPT).
struct InflateArgs {
  const unsigned char* z;
  unsigned char* blob;
  Geometry g;
  long long g0, g1;
  int32_t* status;
  long long zbytes;
};

constexpr int ZI_T = 128;                         // inflate: threads per CTA (one sub-block each)

// Bits of the container from byte `from` on, LSB first, through a 64-bit reservoir refilled
// with aligned 32-bit loads (the last partial word byte by byte); past `end` it reads zeros.
struct RegBits {
  const unsigned char* z;
  long long word;             // next word to load (index of 4-byte words)
  long long end;              // bytes of the container
  unsigned long long buf;
  int nbits;
  long long used;             // bits consumed
  __device__ __forceinline__ void init(const unsigned char* zz, long long from, long long e) {
    z = zz;
    end = e;
    word = from >> 2;
    buf = 0;
    nbits = 0;
    used = 0;
    refill();
    const int skip = (int)(from & 3) * 8;
    buf >>= skip;
    nbits -= skip;
  }
  __device__ __forceinline__ void refill() {
    while (nbits <= 32) {
      unsigned v = 0;
      const long long at = word * 4;
      if (at + 4 <= end) {
        v = __ldg(reinterpret_cast<const unsigned*>(z) + word);
      } else {
        for (int k = 0; k < 4; ++k)
          if (at + k < end) v |= (unsigned)z[at + k] << (8 * k);
      }
      buf |= (unsigned long long)v << nbits;
      nbits += 32;
      ++word;
    }
  }
  __device__ __forceinline__ unsigned peek(int n) { return (unsigned)buf & ((1u << n) - 1u); }
  __device__ __forceinline__ void skip(int n) {
    buf >>= n;
    nbits -= n;
    used += n;
    refill();
  }
  __device__ __forceinline__ unsigned get(int n) {
    const unsigned v = n ? peek(n) : 0u;
    skip(n);
    return v;
  }
};

// Decoded bytes go out as 32-bit words (the raw image starts on a 16-byte boundary); the last
// 16 bytes are kept in registers for matches (this encoder's distances are at most 15).
struct ByteOut {
  unsigned* dst;
  int n;                      // bytes written
  unsigned acc;
  unsigned long long h0, h1;  // h0: the 8 most recent bytes (byte 0 = last), h1: the 8 before
  __device__ __forceinline__ void put(unsigned b) {
    acc |= b << (8 * (n & 3));
    h1 = (h1 << 8) | (h0 >> 56);
    h0 = (h0 << 8) | b;
    ++n;
    if ((n & 3) == 0) { dst[(n >> 2) - 1] = acc; acc = 0; }
  }
  __device__ __forceinline__ unsigned back(int d) const {   // the byte d back (1 <= d <= 16)
    return d <= 8 ? (unsigned)(h0 >> (8 * (d - 1))) & 0xFFu : (unsigned)(h1 >> (8 * (d - 9))) & 0xFFu;
  }
};

// One thread per sub-block (LPT = 1) or one warp per sub-block with only its first lane
// decoding (LPT = 32: no divergence between sub-blocks, for small counts where latency rather
// than throughput matters): inflates the sub-block's DEFLATE data (the fixed-Huffman and stored
// blocks this encoder writes; anything else is NUMARCK_ERR_CORRUPT) into the raw image and
// pads it.
template <int LPT>
__global__ void __launch_bounds__(ZI_T) z4_inflate(InflateArgs A, const int64_t* sub_zoff) {
  const long long tid = (long long)blockIdx.x * ZI_T + threadIdx.x;
  if (tid % LPT) return;
  const long long gt = A.g0 + tid / LPT;
  if (gt > A.g1) return;
  const Geometry& g = A.g;
  const long long q = gt / g.spb, t = gt - q * g.spb;
  const long long j0 = q * g.epb + t * SUB;
  const long long bend = min((long long)g.n, (long long)((q + 1) * g.epb));
  const int cnt = (int)min((long long)SUB, bend - j0);
  const int tb = (cnt * g.B + 7) / 8;
  const int padded = 16 * ((cnt * g.B + 127) / 128);
  unsigned char* dst = A.blob + g.off_index + q * g.block_stride + t * (long long)(SUB / 8 * g.B);
  const long long zo = sub_zoff[gt];
  const long long zend = gt + 1 < g.nsub ? sub_zoff[gt + 1] : A.zbytes;
  int rc = (zo < 0 || zo > zend || zend > A.zbytes) ? NUMARCK_ERR_CORRUPT : 0;
  RegBits br;
  br.init(A.z, rc ? 0 : zo, rc ? 0 : zend);
  const long long limit = rc ? 0 : (zend - zo) * 8;
  ByteOut out{reinterpret_cast<unsigned*>(dst), 0, 0u, 0ull, 0ull};
  const unsigned hdr = rc ? 0u : br.get(3);
  if (!rc && hdr == 0u) {                         // stored: BFINAL 0, BTYPE 00
    br.skip((8 - (int)(br.used & 7)) & 7);        // to the byte boundary
    const unsigned len = br.get(16), nlen = br.get(16);
    if ((len ^ nlen) != 0xFFFFu || (int)len != tb || br.used + 8LL * len > limit) {
      rc = NUMARCK_ERR_CORRUPT;
    } else {
      for (int k = 0; k < tb; ++k) out.put(br.get(8));
    }
  } else if (!rc && hdr != 2u) {                  // neither stored nor BTYPE 01
    rc = NUMARCK_ERR_CORRUPT;
  }
  while (!rc && hdr == 2u) {
    if (br.used > limit) { rc = NUMARCK_ERR_CORRUPT; break; }
    // fixed Huffman literal/length symbol (RFC 1951 §3.2.6)
    const unsigned b9 = br.peek(9);
    int sym;
    const unsigned c7 = rev(b9 & 0x7Fu, 7);
    if (c7 <= 23) {
      sym = 256 + (int)c7;
      br.skip(7);
    } else {
      const unsigned c8 = rev(b9 & 0xFFu, 8);
      if (c8 >= 0x30 && c8 <= 0xBF) { sym = (int)(c8 - 0x30); br.skip(8); }
      else if (c8 >= 0xC0 && c8 <= 0xC7) { sym = 280 + (int)(c8 - 0xC0); br.skip(8); }
      else { sym = 144 + (int)(rev(b9, 9) - 0x190); br.skip(9); }
    }
    if (sym > 285) { rc = NUMARCK_ERR_CORRUPT; break; }
    if (sym < 256) {
      if (out.n >= tb) { rc = NUMARCK_ERR_CORRUPT; break; }
      out.put((unsigned)sym);
    } else if (sym == 256) {
      break;
    } else {
      const int lc = sym - 257;
      const int len = c_len_base[lc] + (int)br.get(c_len_extra[lc]);
      const int dc = (int)rev(br.get(5), 5);
      if (dc > 29) { rc = NUMARCK_ERR_CORRUPT; break; }
      const int d = c_dist_base[dc] + (int)br.get(c_dist_extra[dc]);
      if (d > out.n || out.n + len > tb) { rc = NUMARCK_ERR_CORRUPT; break; }
      if (d <= 16) {
        for (int k = 0; k < len; ++k) out.put(out.back(d));
      } else {                                    // not written by this encoder: from memory
        for (int k = 0; k < len; ++k) {
          const int at = out.n - d;
          const unsigned b = (at >> 2) < (out.n >> 2)
                                 ? (reinterpret_cast<const unsigned*>(dst)[at >> 2] >> (8 * (at & 3))) & 0xFFu
                                 : (out.acc >> (8 * (at & 3))) & 0xFFu;
          out.put(b);
        }
      }
    }
  }
  if (!rc && out.n != tb) rc = NUMARCK_ERR_CORRUPT;
  if (rc) {
    if (A.status) atomicExch(A.status, rc);
    return;
  }
  if (out.n & 3) out.dst[out.n >> 2] = out.acc;   // the last partial word (zero-padded)
  for (int w = (tb + 3) >> 2; w < padded / 4; ++w) out.dst[w] = 0u;
}

}  // namespace

int zindex_layout(const Geometry& g, numarck_zindex_header* zh) {
  std::memset(zh, 0, sizeof(*zh));
  zh->magic = NUMARCK_ZINDEX_MAGIC;
  zh->version = 1;
  zh->B = g.B;
  zh->n = g.n;
  zh->nblocks = g.nblocks;
  zh->nsub = g.nsub;
  zh->off_zoff = NUMARCK_ZINDEX_HEADER_BYTES;
  zh->off_sub_zoff = round_up_i64(zh->off_zoff + (g.nblocks + 1) * 8, 16);
  zh->off_data = round_up_i64(zh->off_sub_zoff + g.nsub * 8, 16);
  return NUMARCK_OK;
}

int64_t zindex_bound(const Geometry& g) {
  numarck_zindex_header zh;
  zindex_layout(g, &zh);
  // every byte a 9-bit literal, plus per sub-block 3 + 7 + 3 bits, padding and 4 bytes, plus
  // per block 2 + 6 bytes
  return zh.off_data + g.index_bytes * 9 / 8 + g.nsub * 10 + g.nblocks * 8 + 64;
}

cudaError_t launch_deflate(const unsigned char* blob, const Geometry& g, unsigned char* z,
                           unsigned char* ws, int sms, cudaStream_t s) {
  if (g.nsub == 0) return cudaSuccess;
  ZArgs A;
  A.blob = blob;
  A.g = g;
  A.z = z;
  zindex_layout(g, &A.zh);
  A.tile_bytes = reinterpret_cast<int64_t*>(ws);
  A.adler_a = reinterpret_cast<unsigned*>(ws + g.nsub * 8);
  A.adler_w = A.adler_a + g.nsub;
  A.lane_bits = reinterpret_cast<unsigned short*>(ws + g.nsub * 16);
  const size_t smem1 = (size_t)ZW * z_in_bytes(g.B);
  const size_t smem3 = smem1 + (size_t)ZW * z_out_words(g.B) * 4;
  static bool configured[64] = {false};   // the largest B's sizes, once per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !configured[dev]) {
    const int max1 = ZW * z_in_bytes(NUMARCK_MAX_B);
    const int max3 = max1 + ZW * z_out_words(NUMARCK_MAX_B) * 4;
    cudaError_t e = cudaFuncSetAttribute(z1_size, cudaFuncAttributeMaxDynamicSharedMemorySize, max1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(z3_write, cudaFuncAttributeMaxDynamicSharedMemorySize, max3);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured[dev] = true;
  }
  long long blocks = (g.nsub + ZW - 1) / ZW;
  if (blocks > (long long)sms * 32) blocks = (long long)sms * 32;
  z1_size<<<(int)blocks, ZT, smem1, s>>>(A);
  z2_scan<<<1, 1024, 0, s>>>(A);
  z3_write<<<(int)blocks, ZT, smem3, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_inflate(const unsigned char* z, long long zbytes, unsigned char* blob,
                           const Geometry& g, long long g0, long long g1, int32_t* status,
                           cudaStream_t s) {
  if (g1 < g0) return cudaSuccess;
  InflateArgs A{z, blob, g, g0, g1, status, zbytes};
  const long long n = g1 - g0 + 1;
  // the sub-block offsets lie at a fixed place of the container (see zindex_layout)
  numarck_zindex_header lay;
  zindex_layout(g, &lay);
  const int64_t* sub_zoff = reinterpret_cast<const int64_t*>(z + lay.off_sub_zoff);
  if (n < 16384)     // few sub-blocks (a partial decompression): one warp each, all SMs busy
    z4_inflate<32><<<(unsigned)((n * 32 + ZI_T - 1) / ZI_T), ZI_T, 0, s>>>(A, sub_zoff);
  else
    z4_inflate<1><<<(unsigned)((n + ZI_T - 1) / ZI_T), ZI_T, 0, s>>>(A, sub_zoff);
  return cudaGetLastError();
}

}  // namespace nmk
