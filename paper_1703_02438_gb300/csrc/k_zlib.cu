// k_zlib.cu — lossless compression of the index table (§IV.C: "NUMARCK splits the index table
// into blocks of same size and compresses each block using the ZLIB"), as zlib streams (RFC
// 1950) of DEFLATE data (RFC 1951) that any inflater reads, and the matching GPU inflater.
//
// Stream layout of index block q (the block's ceil(count * B / 8) bytes, without the 16-byte
// padding of the raw blob):
//   0x78 0x01                                       zlib header (deflate, 32 KB window)
//   for each 4096-element sub-block t of the block, the smallest of:
//     one dynamic-Huffman DEFLATE block (BFINAL 0, BTYPE 10: the index block's code, built from
//     the symbol counts of all its sub-blocks) of t's bytes, then an empty stored block
//     (BFINAL 0, BTYPE 00, LEN 0, NLEN 0xFFFF) that ends t's data on a byte boundary;
//     the same with a fixed-Huffman block (BTYPE 01);
//     one stored block (BFINAL 0, BTYPE 00) holding t's bytes
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
// its codes at its bit offset. The dynamic code of an index block comes from the symbol counts of
// all its sub-blocks by a Huffman construction on one lane after a warp-wide sort; a code longer
// than DEFLATE allows (15 bits, 7 for the code-length code) is rebuilt from halved counts until
// it fits. Every sub-block's dynamic block repeats that code in its own header. Z1 counts the
// fixed-code bits, the symbols and the Adler-32 partial sums, Zb builds each block's code, Zc
// picks each sub-block's smallest coding, Z2 scans the sizes into offsets, Z3 writes the
// streams; Z4 inflates sub-blocks.
#include <algorithm>
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
  unsigned char* kind;       // per sub-block: the block type Z1 chose (0 stored, 1 fixed, 2 dynamic)
  unsigned* counts;          // per index block: literal/length and distance counts (288 + 32)
  struct BlockCode* codes;   // per index block: its dynamic code (Zb)
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

// Greedy parse of bytes [c0, c1) of s with matches at distance p: sink.lit(byte) for a literal,
// sink.match(length code index, length, distance code, distance) for a match, in order.
template <typename Sink>
__device__ void parse_chunk(const unsigned char* s, int c0, int c1, int p, Sink& sink) {
  const int dc = dist_code(p);
  int i = c0;
  while (i < c1) {
    int len = 0;
    if (i >= p) {
      while (i + len < c1 && len < 258 && s[i + len] == s[i + len - p]) ++len;
    }
    if (len >= 3) {
      sink.match(len_code(len), len, dc, p);
      i += len;
    } else {
      sink.lit(s[i]);
      ++i;
    }
  }
}

constexpr int NLL = 286;        // literal/length alphabet (RFC 1951 §3.2.5)
constexpr int ND = 30;          // distance alphabet
constexpr int NCL = 19;         // code-length alphabet (§3.2.7)
// order in which the code-length code's lengths are sent (§3.2.7)
__constant__ unsigned char c_cl_order[NCL] = {16, 17, 18, 0, 8, 7, 9, 6, 10, 5,
                                              11, 4, 12, 3, 13, 2, 14, 1, 15};

// Per-warp state of a dynamic-Huffman block: symbol counts, code lengths and codes of the
// literal/length, distance and code-length alphabets, the run-length coded lengths, and the
// construction's scratch.
struct HuffWarp {
  unsigned fll[288], fd[32], fcl[32];
  unsigned keys[512];                 // (count << 9) | symbol, sorted
  unsigned wt[576];                   // node weights, then depths
  unsigned short par[576];            // node parents
  unsigned short cll[288], cd[32], ccl[32];   // codes, bit-reversed for the LSB-first stream
  unsigned char lll[288], ld[32], lcl[32];    // code lengths
  unsigned char rle_sym[320], rle_ext[320];   // run-length coded lengths (§3.2.7)
  int nrle, hlit, hdist, hclen, hdr_bits;
};

// Code lengths of a Huffman code for counts f[0..n) (n <= 288) into len[], at most maxlen bits:
// the warp sorts (count, symbol) keys, lane 0 merges the two queues of leaves and internal nodes
// (ties: leaf first) and reads the leaves' depths. A code deeper than maxlen is rebuilt from
// counts halved (rounded up) until it fits. Unused symbols get 0; a single used symbol gets 1.
__device__ void huff_lengths(const unsigned* f, int n, int maxlen, unsigned char* len, HuffWarp& h,
                             int lane) {
  const int P = n <= 32 ? 32 : 512;
  for (int shift = 0;; ++shift) {
    for (int i = lane; i < P; i += 32) {
      unsigned key = 0xFFFFFFFFu;
      if (i < n && f[i]) {
        const unsigned c = (f[i] + (1u << shift) - 1u) >> shift;
        key = (c << 9) | (unsigned)i;
      }
      h.keys[i] = key;
    }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {        // bitonic sort, ascending
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int x = i ^ j;
          if (x > i) {
            const unsigned a = h.keys[i], b = h.keys[x];
            if ((a > b) == ((i & k) == 0)) { h.keys[i] = b; h.keys[x] = a; }
          }
        }
        __syncwarp();
      }
    }
    int depth = 0;
    if (lane == 0) {
      for (int i = 0; i < n; ++i) len[i] = 0;
      int m = 0;
      while (m < P && h.keys[m] != 0xFFFFFFFFu) ++m;
      if (m == 1) {
        len[h.keys[0] & 511u] = 1;
        depth = 1;
      } else if (m > 1) {
        for (int i = 0; i < m; ++i) h.wt[i] = h.keys[i] >> 9;
        int li = 0, ii = m, next = m;
        for (int t = 0; t < m - 1; ++t) {
          int ab[2];
          for (int c = 0; c < 2; ++c) {
            if (li < m && (ii >= next || h.wt[li] <= h.wt[ii])) ab[c] = li++;
            else ab[c] = ii++;
          }
          h.wt[next] = h.wt[ab[0]] + h.wt[ab[1]];
          h.par[ab[0]] = (unsigned short)next;
          h.par[ab[1]] = (unsigned short)next;
          ++next;
        }
        const int root = 2 * m - 2;
        h.wt[root] = 0;                         // weights are no longer needed: depths
        for (int id = root - 1; id >= 0; --id) h.wt[id] = h.wt[h.par[id]] + 1;
        for (int i = 0; i < m; ++i) {
          len[h.keys[i] & 511u] = (unsigned char)h.wt[i];
          depth = max(depth, (int)h.wt[i]);
        }
      }
    }
    depth = __shfl_sync(0xffffffffu, depth, 0);
    __syncwarp();
    if (depth <= maxlen) return;
  }
}

// Canonical codes (§3.2.2) of the lengths len[0..n), bit-reversed for the LSB-first stream.
__device__ void canonical_codes(const unsigned char* len, int n, unsigned short* code) {
  int count[16] = {0};
  for (int i = 0; i < n; ++i) count[len[i]]++;
  count[0] = 0;
  int next[16];
  int c = 0;
  for (int b = 1; b < 16; ++b) {
    c = (c + count[b - 1]) << 1;
    next[b] = c;
  }
  for (int i = 0; i < n; ++i)
    code[i] = len[i] ? (unsigned short)rev((unsigned)next[len[i]]++, len[i]) : 0;
}

// The dynamic code of a sub-block from the counts in h.fll / h.fd (the end-of-block symbol
// included): code lengths, the run-length coded lengths, the code-length code, the header's
// bit count and every code. All lanes call.
__device__ void build_dynamic(HuffWarp& h, int lane) {
  huff_lengths(h.fll, NLL, 15, h.lll, h, lane);
  huff_lengths(h.fd, ND, 15, h.ld, h, lane);
  if (lane == 0) {
    h.hlit = NLL;
    while (h.hlit > 257 && h.lll[h.hlit - 1] == 0) --h.hlit;
    h.hdist = ND;
    while (h.hdist > 1 && h.ld[h.hdist - 1] == 0) --h.hdist;
    for (int i = 0; i < 32; ++i) h.fcl[i] = 0;
    // lengths of both codes as one sequence, run-length coded (16: repeat the previous length
    // 3-6 times, 17: 3-10 zeros, 18: 11-138 zeros)
    const int N = h.hlit + h.hdist;
    int nr = 0;
    for (int i = 0; i < N;) {
      const unsigned char cur = i < h.hlit ? h.lll[i] : h.ld[i - h.hlit];
      int run = 1;
      while (i + run < N && (i + run < h.hlit ? h.lll[i + run] : h.ld[i + run - h.hlit]) == cur)
        ++run;
      i += run;
      if (cur == 0) {
        while (run >= 11) {
          const int r = min(run, 138);
          h.rle_sym[nr] = 18; h.rle_ext[nr++] = (unsigned char)(r - 11); run -= r;
        }
        if (run >= 3) { h.rle_sym[nr] = 17; h.rle_ext[nr++] = (unsigned char)(run - 3); run = 0; }
        while (run > 0) { h.rle_sym[nr] = 0; h.rle_ext[nr++] = 0; --run; }
      } else {
        h.rle_sym[nr] = cur; h.rle_ext[nr++] = 0; --run;
        while (run >= 3) {
          const int r = min(run, 6);
          h.rle_sym[nr] = 16; h.rle_ext[nr++] = (unsigned char)(r - 3); run -= r;
        }
        while (run > 0) { h.rle_sym[nr] = cur; h.rle_ext[nr++] = 0; --run; }
      }
    }
    h.nrle = nr;
    int used = 0;
    for (int i = 0; i < nr; ++i) h.fcl[h.rle_sym[i]]++;
    for (int i = 0; i < NCL; ++i) used += h.fcl[i] != 0;
    if (used == 1) h.fcl[h.fcl[0] ? 1 : 0] = 1;   // a one-symbol code-length code is incomplete
  }
  __syncwarp();
  huff_lengths(h.fcl, NCL, 7, h.lcl, h, lane);
  if (lane == 0) {
    h.hclen = NCL;
    while (h.hclen > 4 && h.lcl[c_cl_order[h.hclen - 1]] == 0) --h.hclen;
    int bits = 5 + 5 + 4 + 3 * h.hclen;
    for (int i = 0; i < h.nrle; ++i) {
      const int sym = h.rle_sym[i];
      bits += h.lcl[sym] + (sym == 16 ? 2 : sym == 17 ? 3 : sym == 18 ? 7 : 0);
    }
    h.hdr_bits = bits;
    canonical_codes(h.lll, NLL, h.cll);
    canonical_codes(h.ld, ND, h.cd);
    canonical_codes(h.lcl, NCL, h.ccl);
  }
  __syncwarp();
}

// Sinks of the parse.
struct FixedCount {          // bits of the codes under the fixed Huffman code
  int bits = 0;
  __device__ void lit(unsigned b) { bits += b < 144 ? 8 : 9; }
  __device__ void match(int lc, int, int dc, int) {
    int l;
    fixed_code(257 + lc, &l);
    bits += l + c_len_extra[lc] + 5 + c_dist_extra[dc];
  }
};
struct SymbolCount {         // the warp's symbol counts (shared-memory atomics)
  unsigned* fll;
  unsigned* fd;
  __device__ void lit(unsigned b) { atomicAdd(&fll[b], 1u); }
  __device__ void match(int lc, int, int dc, int) {
    atomicAdd(&fll[257 + lc], 1u);
    atomicAdd(&fd[dc], 1u);
  }
};
struct DynCount {            // bits of the codes under a dynamic code
  const HuffWarp* h;
  int bits = 0;
  __device__ void lit(unsigned b) { bits += h->lll[b]; }
  __device__ void match(int lc, int, int dc, int) {
    bits += h->lll[257 + lc] + c_len_extra[lc] + h->ld[dc] + c_dist_extra[dc];
  }
};
struct FixedWrite {
  LaneBits* bw;
  __device__ void lit(unsigned b) {
    int l;
    const unsigned code = fixed_code(b, &l);
    bw->put(code, l);
  }
  __device__ void match(int lc, int len, int dc, int d) {
    int l;
    const unsigned code = fixed_code(257 + lc, &l);
    bw->put(code, l);
    bw->put((unsigned)(len - c_len_base[lc]), c_len_extra[lc]);
    bw->put(rev((unsigned)dc, 5), 5);
    bw->put((unsigned)(d - c_dist_base[dc]), c_dist_extra[dc]);
  }
};
struct DynWrite {
  LaneBits* bw;
  const HuffWarp* h;
  __device__ void lit(unsigned b) { bw->put(h->cll[b], h->lll[b]); }
  __device__ void match(int lc, int len, int dc, int d) {
    bw->put(h->cll[257 + lc], h->lll[257 + lc]);
    bw->put((unsigned)(len - c_len_base[lc]), c_len_extra[lc]);
    bw->put(h->cd[dc], h->ld[dc]);
    bw->put((unsigned)(d - c_dist_base[dc]), c_dist_extra[dc]);
  }
};

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

// The dynamic code of one index block (built once from the counts of all its sub-blocks and
// used by each of them; every sub-block's DEFLATE block still carries the code in its own
// header, so that it inflates on its own).
struct BlockCode {
  unsigned short cll[288], cd[32], ccl[32];
  unsigned char lll[288], ld[32], lcl[32];
  unsigned char rle_sym[320], rle_ext[320];
  int nrle, hlit, hdist, hclen, hdr_bits;
};

// Copies a block's code into (all = false: only the code lengths) the warp's state.
__device__ __forceinline__ void load_code(const BlockCode& c, HuffWarp& h, int lane, bool all) {
  for (int i = lane; i < 288; i += 32) h.lll[i] = c.lll[i];
  h.ld[lane] = c.ld[lane];
  if (all) {
    for (int i = lane; i < 288; i += 32) h.cll[i] = c.cll[i];
    h.cd[lane] = c.cd[lane];
    h.ccl[lane] = c.ccl[lane];
    h.lcl[lane] = c.lcl[lane];
    for (int i = lane; i < 320; i += 32) {
      h.rle_sym[i] = c.rle_sym[i];
      h.rle_ext[i] = c.rle_ext[i];
    }
    if (lane == 0) {
      h.nrle = c.nrle; h.hlit = c.hlit; h.hdist = c.hdist; h.hclen = c.hclen;
      h.hdr_bits = c.hdr_bits;
    }
  }
  __syncwarp();
}

// Bytes of a sub-block's dynamic-Huffman data: block header (3 bits), the code's header, the
// codes, end of block, then the empty stored block (3 bits, padding, 4 bytes).
__device__ __forceinline__ int dynamic_bytes(const HuffWarp& h, int code_bits) {
  return (3 + h.hdr_bits + code_bits + h.lll[256] + 3 + 7) / 8 + 4;
}

// Counting sink for Z1's parse: fixed-code bits and the symbol counts at once.
struct FixedAndCount {
  FixedCount fc;
  SymbolCount sc;
  __device__ void lit(unsigned b) { fc.lit(b); sc.lit(b); }
  __device__ void match(int lc, int len, int dc, int d) {
    fc.match(lc, len, dc, d);
    sc.match(lc, len, dc, d);
  }
};

// Z1: per sub-block, each lane's code bits under the fixed code, the sub-block's symbol counts
// (added into its index block's counts, end of block included) and the Adler-32 partial sums.
__global__ void __launch_bounds__(ZT) z1_count(ZArgs A) {
  extern __shared__ __align__(16) unsigned char z_smem[];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int p = period_of(A.g.B);
  unsigned char* s = z_smem + warp * z_in_bytes(A.g.B);
  HuffWarp& h = reinterpret_cast<HuffWarp*>(z_smem + ZW * z_in_bytes(A.g.B))[warp];
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.padded / 16; i += 32)
      reinterpret_cast<uint4*>(s)[i] = __ldg(reinterpret_cast<const uint4*>(z.src) + i);
    for (int i = lane; i < 288; i += 32) h.fll[i] = 0u;
    h.fd[lane] = 0u;
    __syncwarp();
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    FixedAndCount fac{FixedCount{}, SymbolCount{h.fll, h.fd}};
    parse_chunk(s, c0, c1, p, fac);
    A.lane_bits[gt * 32 + lane] = (unsigned short)fac.fc.bits;
    __syncwarp();
    unsigned* bc = A.counts + z.q * 320;
    for (int i = lane; i < 288; i += 32)
      if (h.fll[i]) atomicAdd(&bc[i], h.fll[i]);
    if (h.fd[lane]) atomicAdd(&bc[288 + lane], h.fd[lane]);
    if (lane == 0) atomicAdd(&bc[256], 1u);        // the sub-block's end of block
    unsigned a = 0;
    unsigned long long w = 0;
    for (int i = lane; i < z.tb; i += 32) {
      a += s[i];
      w += (unsigned long long)(z.tb - i) * s[i];
    }
    a = __reduce_add_sync(0xffffffffu, a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) {
      A.adler_a[gt] = a % ADLER;
      A.adler_w[gt] = (unsigned)(w % ADLER);
    }
    __syncwarp();
  }
}

// Zb: the dynamic code of each index block from its counts (one warp per block); the counts are
// left zero for the next call.
__global__ void __launch_bounds__(ZT) zb_build(ZArgs A) {
  extern __shared__ __align__(16) unsigned char z_smem[];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  HuffWarp& h = reinterpret_cast<HuffWarp*>(z_smem)[warp];
  for (long long q = (long long)blockIdx.x * ZW + warp; q < A.g.nblocks;
       q += (long long)gridDim.x * ZW) {
    unsigned* bc = A.counts + q * 320;
    for (int i = lane; i < 288; i += 32) { h.fll[i] = bc[i]; bc[i] = 0u; }
    h.fd[lane] = bc[288 + lane];
    bc[288 + lane] = 0u;
    __syncwarp();
    build_dynamic(h, lane);
    BlockCode& c = A.codes[q];
    for (int i = lane; i < 288; i += 32) { c.lll[i] = h.lll[i]; c.cll[i] = h.cll[i]; }
    c.ld[lane] = h.ld[lane];
    c.cd[lane] = h.cd[lane];
    c.lcl[lane] = h.lcl[lane];
    c.ccl[lane] = h.ccl[lane];
    for (int i = lane; i < 320; i += 32) { c.rle_sym[i] = h.rle_sym[i]; c.rle_ext[i] = h.rle_ext[i]; }
    if (lane == 0) {
      c.nrle = h.nrle; c.hlit = h.hlit; c.hdist = h.hdist; c.hclen = h.hclen;
      c.hdr_bits = h.hdr_bits;
    }
    __syncwarp();
  }
}

// Zc: per sub-block, its bits under its block's dynamic code; the smallest coding (stored,
// fixed or dynamic Huffman) and its slot size, and each lane's code bits under that coding.
__global__ void __launch_bounds__(ZT) zc_choose(ZArgs A) {
  extern __shared__ __align__(16) unsigned char z_smem[];
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int p = period_of(A.g.B);
  unsigned char* s = z_smem + warp * z_in_bytes(A.g.B);
  HuffWarp& h = reinterpret_cast<HuffWarp*>(z_smem + ZW * z_in_bytes(A.g.B))[warp];
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.padded / 16; i += 32)
      reinterpret_cast<uint4*>(s)[i] = __ldg(reinterpret_cast<const uint4*>(z.src) + i);
    load_code(A.codes[z.q], h, lane, false);
    if (lane == 0) h.hdr_bits = A.codes[z.q].hdr_bits;
    __syncwarp();
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    DynCount dcount{&h};
    parse_chunk(s, c0, c1, p, dcount);
    const int fbits = A.lane_bits[gt * 32 + lane];
    const int ftotal = __reduce_add_sync(0xffffffffu, fbits);
    const int dtotal = __reduce_add_sync(0xffffffffu, dcount.bits);
    const int fb = fixed_bytes(ftotal), db = dynamic_bytes(h, dtotal), sb = stored_bytes(z.tb);
    const int kind = (fb <= sb && fb <= db) ? 1 : (db < sb ? 2 : 0);
    A.lane_bits[gt * 32 + lane] = (unsigned short)(kind == 2 ? dcount.bits : fbits);
    if (lane == 0) {
      A.kind[gt] = (unsigned char)kind;
      A.tile_bytes[gt] = slot_bytes(kind == 1 ? fb : kind == 2 ? db : sb, z.first, z.last);
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
  HuffWarp& h = reinterpret_cast<HuffWarp*>(z_smem + ZW * inb + ZW * outw * 4)[warp];
  for (long long gt = (long long)blockIdx.x * ZW + warp; gt < A.g.nsub;
       gt += (long long)gridDim.x * ZW) {
    const ZTile z = ztile(A, gt);
    for (int i = lane; i < z.padded / 16; i += 32)
      reinterpret_cast<uint4*>(s)[i] = __ldg(reinterpret_cast<const uint4*>(z.src) + i);
    const int per = (z.tb + 31) / 32;
    const int c0 = min(z.tb, lane * per), c1 = min(z.tb, c0 + per);
    const int kind = A.kind[gt];
    const int bits = A.lane_bits[gt * 32 + lane];    // Z1's count of this lane's code bits
    int incl = bits;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (kind == 2) load_code(A.codes[z.q], h, lane, true);   // the block's code (Zb)
    const int hdr = kind == 2 ? h.hdr_bits : 0;
    // the words the codes (block headers, codes, end of block, stored-block header bits) touch
    const int used_words = (3 + hdr + total + 15 + 3 + 31) / 32 + 1;
    for (int i = lane; i < used_words; i += 32) o[i] = 0u;
    __syncwarp();
    const long long off = A.tile_bytes[gt];
    unsigned char* dst = A.z + off;
    const int k = z.first ? 2 : 0;
    if (z.first && lane == 0) { dst[0] = 0x78; dst[1] = 0x01; }
    int nb;                                // bytes of the sub-block's DEFLATE data
    if (kind == 0) {
      // stored block: BFINAL 0, BTYPE 00 (the rest of the header byte is padding), LEN, NLEN
      if (lane == 0) {
        dst[k] = 0x00;
        dst[k + 1] = (unsigned char)z.tb; dst[k + 2] = (unsigned char)(z.tb >> 8);
        dst[k + 3] = (unsigned char)~z.tb; dst[k + 4] = (unsigned char)(~z.tb >> 8);
      }
      for (int i = lane; i < z.tb; i += 32) dst[k + 5 + i] = s[i];
      nb = stored_bytes(z.tb);
    } else {
      LaneBits bw(o, 3 + hdr + incl - bits);
      if (lane == 0) {
        BitWriter hw{o, 0};
        if (kind == 1) {
          hw.put(2u, 3);                     // BFINAL 0, BTYPE 01 (fixed Huffman)
        } else {
          hw.put(4u, 3);                     // BFINAL 0, BTYPE 10 (dynamic Huffman)
          hw.put((unsigned)(h.hlit - 257), 5);
          hw.put((unsigned)(h.hdist - 1), 5);
          hw.put((unsigned)(h.hclen - 4), 4);
          for (int i = 0; i < h.hclen; ++i) hw.put(h.lcl[c_cl_order[i]], 3);
          for (int i = 0; i < h.nrle; ++i) {
            const int sym = h.rle_sym[i];
            hw.put(h.ccl[sym], h.lcl[sym]);
            if (sym >= 16) hw.put(h.rle_ext[i], sym == 16 ? 2 : sym == 17 ? 3 : 7);
          }
        }
      }
      if (kind == 1) {
        FixedWrite fw{&bw};
        parse_chunk(s, c0, c1, p, fw);
      } else {
        DynWrite dw{&bw, &h};
        parse_chunk(s, c0, c1, p, dw);
      }
      bw.flush();
      __syncwarp();
      int end_bits = 3 + hdr + total;
      const int eob = kind == 1 ? 7 : h.lll[256];
      if (lane == 0) {
        BitWriter ew{o, end_bits};
        ew.put(kind == 1 ? 0u : h.cll[256], eob);   // end of block (symbol 256)
        ew.put(0u, 3);                       // BFINAL 0, BTYPE 00 (stored), LEN 0 follows
      }
      __syncwarp();
      end_bits += eob + 3;
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

// Z4: inflate sub-blocks [g0, g1] back into the raw index section of a blob (the blocks this
// encoder writes; anything else is reported as NUMARCK_ERR_CORRUPT).
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

// A canonical Huffman decoder (RFC 1951 §3.2.2): the number of codes of each length and the
// symbols in code order. decode() walks the lengths one bit at a time from the 15 bits it peeks
// (the codes arrive most significant bit first within the LSB-first stream).
struct HuffDec {
  unsigned short count[16];
  unsigned short sym[288];
  // Builds the decoder of lengths len[0..n); returns false if the code is over-subscribed, or
  // incomplete unless `partial_ok` and it has a single code of length 1 (a distance code
  // with one used distance) or no code at all.
  __device__ bool build(const unsigned char* len, int n, bool partial_ok) {
    for (int b = 0; b < 16; ++b) count[b] = 0;
    for (int i = 0; i < n; ++i) count[len[i]]++;
    unsigned short offs[16];
    int left = 1;
    for (int b = 1; b < 16; ++b) {
      left <<= 1;
      left -= count[b];
      if (left < 0) return false;                 // over-subscribed
    }
    offs[1] = 0;
    for (int b = 1; b < 15; ++b) offs[b + 1] = offs[b] + count[b];
    for (int i = 0; i < n; ++i)
      if (len[i]) sym[offs[len[i]]++] = (unsigned short)i;
    const int used = n - count[0];
    if (left > 0 && !(partial_ok && (used == 0 || (used == 1 && count[1] == 1)))) return false;
    return true;
  }
  // The next symbol, or -1 for a bit pattern that is no code.
  __device__ int decode(RegBits& br) const {
    const unsigned bits = br.peek(15);
    int code = 0, first = 0, index = 0;
    for (int len = 1; len < 16; ++len) {
      code |= (int)((bits >> (len - 1)) & 1u);
      const int c = count[len];
      if (code - first < c) {
        br.skip(len);
        return sym[index + code - first];
      }
      index += c;
      first = (first + c) << 1;
      code <<= 1;
    }
    return -1;
  }
};

// The header of a dynamic-Huffman block (after its 3 block-header bits): the literal/length and
// distance decoders. Returns 0 or NUMARCK_ERR_CORRUPT.
__device__ int read_dynamic_header(RegBits& br, long long limit, HuffDec& ll, HuffDec& dd) {
  const int hlit = (int)br.get(5) + 257, hdist = (int)br.get(5) + 1, hclen = (int)br.get(4) + 4;
  if (hlit > NLL || hdist > ND) return NUMARCK_ERR_CORRUPT;
  unsigned char lens[NLL + ND];
  unsigned char cl[NCL];
  for (int i = 0; i < NCL; ++i) cl[i] = 0;
  for (int i = 0; i < hclen; ++i) cl[c_cl_order[i]] = (unsigned char)br.get(3);
  HuffDec& cd = dd;                               // the distance decoder's storage, for now
  if (!cd.build(cl, NCL, false)) return NUMARCK_ERR_CORRUPT;
  const int N = hlit + hdist;
  for (int i = 0; i < N;) {
    if (br.used > limit) return NUMARCK_ERR_CORRUPT;
    const int sym = cd.decode(br);
    if (sym < 0) return NUMARCK_ERR_CORRUPT;
    if (sym < 16) {
      lens[i++] = (unsigned char)sym;
      continue;
    }
    int rep, val = 0;
    if (sym == 16) {
      if (i == 0) return NUMARCK_ERR_CORRUPT;
      val = lens[i - 1];
      rep = 3 + (int)br.get(2);
    } else if (sym == 17) {
      rep = 3 + (int)br.get(3);
    } else {
      rep = 11 + (int)br.get(7);
    }
    if (i + rep > N) return NUMARCK_ERR_CORRUPT;
    while (rep--) lens[i++] = (unsigned char)val;
  }
  if (lens[256] == 0) return NUMARCK_ERR_CORRUPT;     // no end-of-block code
  if (!ll.build(lens, hlit, false)) return NUMARCK_ERR_CORRUPT;
  if (!dd.build(lens + hlit, hdist, true)) return NUMARCK_ERR_CORRUPT;
  return 0;
}

// One thread per sub-block (LPT = 1) or one warp per sub-block with only its first lane
// decoding (LPT = 32: no divergence between sub-blocks, for small counts where latency rather
// than throughput matters): inflates the sub-block's DEFLATE data (one stored, fixed-Huffman or
// dynamic-Huffman block as this encoder writes it; anything else is NUMARCK_ERR_CORRUPT) into the
// raw image and pads it.
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
  } else if (!rc && hdr != 2u && hdr != 4u) {     // neither stored, BTYPE 01 nor BTYPE 10
    rc = NUMARCK_ERR_CORRUPT;
  }
  const bool dynamic = hdr == 4u;
  HuffDec ll, dd;
  if (!rc && dynamic) rc = read_dynamic_header(br, limit, ll, dd);
  while (!rc && (hdr == 2u || hdr == 4u)) {
    if (br.used > limit) { rc = NUMARCK_ERR_CORRUPT; break; }
    int sym;
    if (dynamic) {
      sym = ll.decode(br);
      if (sym < 0) { rc = NUMARCK_ERR_CORRUPT; break; }
    } else {
      // fixed Huffman literal/length symbol (RFC 1951 §3.2.6)
      const unsigned b9 = br.peek(9);
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
      const int dc = dynamic ? dd.decode(br) : (int)rev(br.get(5), 5);
      if (dc < 0 || dc > 29) { rc = NUMARCK_ERR_CORRUPT; break; }
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

int64_t zindex_workspace(const Geometry& g) {
  // per sub-block: slot size/offset (8), Adler-32 sums (8), 32 lanes' code bits (64), kind (1);
  // per index block: symbol counts (320 words) and its dynamic code
  return round_up_i64(g.nsub * 81, 256) + round_up_i64(g.nblocks * 320 * 4, 256) +
         g.nblocks * (int64_t)sizeof(BlockCode) + 256;
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
  A.kind = ws + g.nsub * 80;
  const int64_t cbase = round_up_i64(g.nsub * 81, 256);
  A.counts = reinterpret_cast<unsigned*>(ws + cbase);
  A.codes = reinterpret_cast<BlockCode*>(ws + cbase + round_up_i64(g.nblocks * 320 * 4, 256));
  const size_t huff = (size_t)ZW * sizeof(HuffWarp);
  const size_t smem1 = (size_t)ZW * z_in_bytes(g.B) + huff;
  const size_t smem3 = (size_t)ZW * z_in_bytes(g.B) + (size_t)ZW * z_out_words(g.B) * 4 + huff;
  static bool configured[64] = {false};   // the largest B's sizes, once per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !configured[dev]) {
    const int max1 = ZW * z_in_bytes(NUMARCK_MAX_B) + (int)huff;
    const int max3 = max1 + ZW * z_out_words(NUMARCK_MAX_B) * 4;
    cudaError_t e = cudaFuncSetAttribute(z1_count, cudaFuncAttributeMaxDynamicSharedMemorySize, max1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(zc_choose, cudaFuncAttributeMaxDynamicSharedMemorySize, max1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(zb_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)huff);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(z3_write, cudaFuncAttributeMaxDynamicSharedMemorySize, max3);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured[dev] = true;
  }
  long long blocks = (g.nsub + ZW - 1) / ZW;
  if (blocks > (long long)sms * 32) blocks = (long long)sms * 32;
  // the per-block counts start at zero (Zb leaves them so for the next call)
  if (cudaMemsetAsync(A.counts, 0, (size_t)g.nblocks * 320 * 4, s) != cudaSuccess)
    return cudaGetLastError();
  z1_count<<<(int)blocks, ZT, smem1, s>>>(A);
  long long bblocks = (g.nblocks + ZW - 1) / ZW;
  if (bblocks > (long long)sms * 32) bblocks = (long long)sms * 32;
  zb_build<<<(int)bblocks, ZT, huff, s>>>(A);
  zc_choose<<<(int)blocks, ZT, smem1, s>>>(A);
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
