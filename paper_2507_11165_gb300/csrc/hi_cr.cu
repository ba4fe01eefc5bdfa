// hi_cr.cu -- the compression-ratio-mode lossless pipeline HF-RRE4-TCMS8-RZE1
// of cuSZ-Hi (arXiv 2507.11165, Sec. 5.2.3) over a byte sequence (the
// reordered quantization codes), and its inverse.  The paper names the
// stages; the code construction, block sizes and container are this
// library's reading:
//   HF     Huffman code lengths from the tree that merges the two
//          lowest-ranked live nodes, ranked by (weight, creation index):
//          leaves are created first in symbol order, internal nodes are
//          numbered on as they are formed (a lone symbol gets one bit);
//          while a length exceeds 16 every nonzero weight w becomes
//          max(1, w >> 1) and the tree is built again.  Canonical codes
//          (per length, the first code follows from the counts of the
//          shorter lengths; within a length, symbol order).  Symbols are
//          coded in blocks of 4096, most significant bit first, each block
//          padded with zero bits to a multiple of 32.
//   RRE4   per 16 KiB chunk of the HF bytes: word bitmap (bit i = word i
//          differs from word i - 1, word -1 = 0), LSB first, reduced by
//          RRE1 levels until a level has at most 64 bytes; output = top
//          level | kept bytes of the levels below, top down | kept words.
//   TCMS8  every whole little-endian 8-byte word t of that output becomes
//          (t << 1) ^ (t >> 63) (arithmetic shift); tail bytes stay.
//   RZE1   levels v_0 = those bytes, v_{r+1} = bitmap of (v_r[i] != 0),
//          until a level has at most 64 bytes; payload = top level |
//          nonzero bytes of each level below, top down.  A chunk whose
//          payload would be longer than the chunk is stored raw.
//   stream u64 n | u32 4096 | u32 nblocks | u64 H | u32 16384 | u32 nchunks
//          | u8 length[256] | u32 words[nblocks] | u16 sub[3 nblocks] | zero
//          pad to 4 | (u32 size, u32 m1)[nchunks] | zero pad to 16 |
//          payloads, each padded to 16 (size = padded bytes, bit 31 = raw;
//          m1 = RRE4 output bytes, 0 if raw); sub[3 b + j - 1] = the bit
//          offset in block b of its symbol 1024 j, or its bit count when
//          the block is shorter.
// Encoding: a histogram pass; the code book in one CTA; a warp per HF block
// counting its bits, a scan of the block sizes, a warp per block packing its
// codes (shared-memory words, OR-ed at the lanes' seams); a CTA per 16 KiB
// chunk running RRE4 / TCMS8 / RZE1 in shared memory into a scratch slot; a
// scan of the payload sizes; a gather.  Decoding: a scan of both tables, a
// CTA per chunk expanding the levels (kept byte of rank popcount(bitmap
// [0..i])), a thread per quarter of an HF block decoding its 1024 symbols
// from the block's starting point through a 12-bit table (longer codes by
// comparison), checked to end at the next starting point.
#include <algorithm>

#include "hi_internal.h"
#include "hi_device.cuh"

namespace hi {

constexpr uint32_t kHfBlock = 4096;
constexpr int kHfLmax = 16;
constexpr int kHfLut = 12;  // decode table bits (codes up to this long take one lookup)
constexpr uint32_t kCrChunk = 16384;
constexpr uint32_t kCrRaw = 0x80000000u;
constexpr int kCrThreads = 256;
constexpr uint32_t kCrHdr = 288;  // fixed header + length table
constexpr uint32_t kHfSub = 1024;  // symbols between a block's starting points

__host__ __device__ inline uint64_t cr_nblocks(uint64_t n) { return (n + kHfBlock - 1) / kHfBlock; }
// HF bytes at most: 16 bits a symbol, plus a padding word a block
__host__ __device__ inline uint64_t cr_hmax(uint64_t n) { return 2 * n + 4 * cr_nblocks(n); }
__host__ __device__ inline uint64_t cr_ncmax(uint64_t n) { return (cr_hmax(n) + kCrChunk - 1) / kCrChunk; }
// The chunk table follows the word table and the starting points (3 u16 a
// block, padded to 4 bytes).
__host__ __device__ inline uint64_t cr_tab_off(uint64_t nb) { return kCrHdr + 4 * nb + (6 * nb + 3) / 4 * 4; }
__host__ __device__ inline uint64_t cr_header_bytes(uint64_t nb, uint64_t nc)
{
    return (cr_tab_off(nb) + 8 * nc + 15) / 16 * 16;
}

// Workspace layout (byte offsets, 16-byte aligned).
struct CrWs {
    uint64_t hist, book, hdr, words, woff, psize, pm1, poff, hf, slots, total;
};

__host__ __device__ inline uint64_t a16(uint64_t b) { return (b + 15) / 16 * 16; }

__host__ __device__ inline CrWs cr_ws(uint64_t n)
{
    const uint64_t nb = cr_nblocks(n), nc = cr_ncmax(n);
    CrWs w;
    w.hist = 0;                           // u32[256]
    w.book = w.hist + 1024;               // u8 len[256] | u32 code[256]
    w.hdr = w.book + 256 + 1024;          // u64 H | u32 nchunks | u32 status
    w.words = a16(w.hdr + 16);            // u32[nb]
    w.woff = a16(w.words + 4 * nb);       // u32[nb] (words before the block)
    w.psize = a16(w.woff + 4 * nb);       // u32[nc]
    w.pm1 = a16(w.psize + 4 * nc);        // u32[nc]
    w.poff = a16(w.pm1 + 4 * nc);         // u64[nc]
    w.hf = a16(w.poff + 8 * nc);          // HF bytes
    w.slots = a16(w.hf + cr_hmax(n) + 16);  // kCrChunk bytes a chunk
    w.total = w.slots + nc * kCrChunk;
    return w;
}

// ---------------------------------------------------------------------------
// Shared helpers
// ---------------------------------------------------------------------------
// Exclusive prefix over the block of one count per thread; *total = the sum.
// Two arrays of a word per warp, used by alternate calls (parity), so one
// barrier per call suffices.
__device__ __forceinline__ uint32_t cr_exscan(uint32_t c, uint32_t* s_red, int& parity, uint32_t* total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t* part = s_red + (parity ? 32 : 0);
    parity ^= 1;
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl += t;
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    uint32_t before = 0, tot = 0;
    for (uint32_t w = 0; w < nw; ++w) {
        const uint32_t v = part[w];
        before += (w < warp) ? v : 0u;
        tot += v;
    }
    *total = tot;
    return before + incl - c;
}

// Bit k (k < 4) set when byte k of w is nonzero (exact, no carry between bytes).
__device__ __forceinline__ uint32_t nz_flags4(uint32_t w)
{
    const uint32_t nz = (((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;
    return (((nz >> 7) * 0x00204081u) >> 21) & 0xfu;
}

// Bit k (k < 4) set when byte k of w differs from the byte before it (prev:
// the word before w).
__device__ __forceinline__ uint32_t rep_flags4(uint32_t w, uint32_t prev)
{
    return nz_flags4(w ^ __funnelshift_l(prev, w, 8));
}

// Flags of the 64 bytes v[a .. a + 64) (zero: nonzero bytes; else: bytes
// that differ from their predecessor, v[-1] = 0), cleared at and past L.
// v is 4-byte aligned and readable up to a + 64.
__device__ __forceinline__ uint64_t span_flags(const uint8_t* v, uint32_t a, uint32_t L, bool zero)
{
    uint32_t prev = a ? (uint32_t)v[a - 1] << 24 : 0u;
    uint64_t f = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t w = reinterpret_cast<const uint32_t*>(v + a)[k];
        f |= (uint64_t)(zero ? nz_flags4(w) : rep_flags4(w, prev)) << (4 * k);
        prev = w;
    }
    if (a + 64 > L) {
        const uint32_t valid = L > a ? L - a : 0u;
        f &= valid >= 64 ? ~0ull : ((1ull << valid) - 1ull);
    }
    return f;
}

struct CrLevels {
    uint32_t L[8];
    int R;
};

__host__ __device__ inline CrLevels cr_levels(uint32_t L0)
{
    CrLevels T;
    T.L[0] = L0;
    T.R = 0;
    while (T.L[T.R] > 64 && T.R < 7) {
        T.L[T.R + 1] = (T.L[T.R] + 7) / 8;
        ++T.R;
    }
    return T;
}

// Bitmap level r + 1 of level r (L bytes at v, zero padded to a multiple of
// 64 and readable there) into bm (8 bytes a span); returns the kept count.
__device__ __forceinline__ uint32_t level_bitmap(const uint8_t* v, uint32_t L, uint8_t* bm, bool zero,
                                                 uint32_t* s_red, int& parity)
{
    uint32_t kept = 0;
    for (uint32_t a0 = 0; a0 < L; a0 += 64 * blockDim.x) {
        const uint32_t a = a0 + 64 * threadIdx.x;
        uint64_t f = 0;
        if (a < L) {
            f = span_flags(v, a, L, zero);
            reinterpret_cast<uint2*>(bm)[a / 64] = make_uint2((uint32_t)f, (uint32_t)(f >> 32));
        }
        uint32_t tot;
        cr_exscan((uint32_t)__popcll(f), s_red, parity, &tot);
        kept += tot;
    }
    return kept;
}

// The kept bytes of level v (L bytes) under its bitmap bm, in order, to
// dst + off; returns off + their count.
__device__ __forceinline__ uint32_t level_kept(const uint8_t* v, uint32_t L, const uint8_t* bm, uint8_t* dst,
                                               uint32_t off, uint32_t* s_red, int& parity)
{
    for (uint32_t a0 = 0; a0 < L; a0 += 64 * blockDim.x) {
        const uint32_t a = a0 + 64 * threadIdx.x;
        uint64_t f = 0;
        if (a < L) {
            const uint2 b = reinterpret_cast<const uint2*>(bm)[a / 64];
            f = (uint64_t)b.x | ((uint64_t)b.y << 32);
        }
        uint32_t tot;
        uint32_t pos = off + cr_exscan((uint32_t)__popcll(f), s_red, parity, &tot);
        while (f) {
            const int i = __ffsll((long long)f) - 1;
            f &= f - 1;
            dst[pos++] = v[a + i];
        }
        off += tot;
    }
    return off;
}

// ---------------------------------------------------------------------------
// Encode
// ---------------------------------------------------------------------------
// 256-bin histogram: bytes 126..129 (the bulk of quantization codes) in
// 8-bit counters of one register per thread, folded before they can wrap;
// others by shared-memory reductions.
__global__ void __launch_bounds__(256) k_cr_hist(const uint8_t* __restrict__ in, uint64_t n,
                                                 uint32_t* __restrict__ hist)
{
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    uint32_t hacc = 0;
    int since = 0;
    const uint64_t nv = n / 16;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(in) + i);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t c = (w[j] >> (8 * b)) & 0xffu;
                const uint32_t sh8 = 8u * c - 8u * 126u;
                hacc += __funnelshift_lc(0u, 1u, sh8);
                if (sh8 >= 32u) atomicAdd(&sh[c], 1u);
            }
        if (++since == 15) {  // at most 240 counts a bin: fold before 255
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t v = (hacc >> (8 * b)) & 0xffu;
                if (v) atomicAdd(&sh[126 + b], v);
            }
            hacc = 0;
            since = 0;
        }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t v = (hacc >> (8 * b)) & 0xffu;
        if (v) atomicAdd(&sh[126 + b], v);
    }
    if (blockIdx.x == 0)  // the tail bytes past the last whole vector
        for (uint64_t i = nv * 16 + threadIdx.x; i < n; i += blockDim.x) atomicAdd(&sh[in[i]], 1u);
    __syncthreads();
    const uint32_t v = sh[threadIdx.x];
    if (v) atomicAdd(&hist[threadIdx.x], v);
}

// The code book (one CTA of 8 warps).  Halving every weight k times gives
// max(1, w >> k), so the trees of eight values of k are built at once, one
// per warp, and the first k whose longest code fits in 16 bits is taken --
// the same k as halving one step at a time.  In each warp: ranks of the
// leaves by (weight, symbol), the two-queue Huffman construction by lane 0
// (leaves sorted in one queue, internal nodes in creation order in the other,
// whose weights never decrease; the lighter front first, a leaf on a tie:
// the (weight, creation index) order), then every leaf's depth by walking up
// to the root.  Canonical codes from the lengths.  Writes the lengths into
// the stream header as well.
constexpr int kBookWarps = 8;
__global__ void __launch_bounds__(32 * kBookWarps) k_cr_codebook(const uint32_t* __restrict__ hist,
                                                                 uint8_t* __restrict__ len_out,
                                                                 uint32_t* __restrict__ code_out,
                                                                 uint8_t* __restrict__ hdr_len)
{
    __shared__ uint32_t wkv[kBookWarps][256], lw[kBookWarps][256];  // leaf weights fit 32 bits
    __shared__ uint64_t iw[kBookWarps][256];
    __shared__ uint8_t lsym[kBookWarps][256], lpar[kBookWarps][256], ipar[kBookWarps][256], wlen[kBookWarps][256];
    __shared__ uint32_t h[256];
    __shared__ uint8_t len[256];
    __shared__ uint32_t cnt[kHfLmax + 2], first[kHfLmax + 2];
    __shared__ unsigned s_pick;
    const int t = threadIdx.x, lane = t & 31, g = t >> 5;
    h[t] = hist[t];
    __syncthreads();
    int k = 0;  // symbols present
    for (int s = 0; s < 256; ++s) k += h[s] > 0 ? 1 : 0;
    for (int kb = 0;; kb += kBookWarps) {
        const int shift = kb + g;  // this warp's number of halvings
        for (int v = lane; v < 256; v += 32) {
            const uint32_t hv = h[v];
            wkv[g][v] = hv == 0 ? 0u : (shift >= 32 ? 1u : ((hv >> shift) ? (hv >> shift) : 1u));
        }
        __syncwarp();
        for (int v = lane; v < 256; v += 32) {
            const uint32_t wt = wkv[g][v];
            wlen[g][v] = 0;
            if (wt == 0) continue;
            int r = 0;
            for (int s = 0; s < 256; ++s) {
                const uint32_t ws = wkv[g][s];
                r += (ws != 0 && (ws < wt || (ws == wt && s < v))) ? 1 : 0;
            }
            lw[g][r] = wt;
            lsym[g][r] = (uint8_t)v;
        }
        __syncwarp();
        int n2 = 0;
        if (lane == 0 && k > 1) {
            int i1 = 0, i2 = 0;
            uint64_t fl = lw[g][0], fi = 0;
            for (int step = 0; step < k - 1; ++step) {
                uint64_t sum = 0;
#pragma unroll
                for (int pick = 0; pick < 2; ++pick) {
                    if (i1 < k && (i2 >= n2 || fl <= fi)) {
                        lpar[g][i1] = (uint8_t)n2;
                        sum += fl;
                        ++i1;
                        fl = i1 < k ? lw[g][i1] : 0;
                    } else {
                        ipar[g][i2] = (uint8_t)n2;
                        sum += fi;
                        ++i2;
                        fi = i2 < n2 ? iw[g][i2] : 0;
                    }
                }
                iw[g][n2] = sum;
                if (i2 == n2) fi = sum;  // the internal queue was empty: this node is its front
                ++n2;
            }
        }
        n2 = __shfl_sync(0xffffffffu, n2, 0);
        __syncwarp();
        int mx = 0;
        if (k == 1) {
            if (lane == 0) wlen[g][lsym[g][0]] = 1;
            mx = 1;
        } else {
            for (int i = lane; i < k; i += 32) {
                int j = lpar[g][i], d = 1;
                while (j != n2 - 1) {
                    j = ipar[g][j];
                    ++d;
                }
                wlen[g][lsym[g][i]] = (uint8_t)d;
                mx = d > mx ? d : mx;
            }
        }
        mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)mx);
        if (t == 0) s_pick = 0xffffffffu;
        __syncthreads();
        if (lane == 0 && mx <= kHfLmax) atomicMin(&s_pick, (unsigned)g);
        __syncthreads();
        const unsigned pick = s_pick;
        if (pick != 0xffffffffu) {
            len[t] = wlen[pick][t];
            break;
        }
        __syncthreads();
    }
    __syncthreads();
    // canonical codes: first code of each length from the counts of the shorter ones
    if (t <= kHfLmax + 1) cnt[t] = 0;
    __syncthreads();
    const int l = len[t];
    if (l) atomicAdd(&cnt[l], 1u);
    __syncthreads();
    if (t == 0) {
        uint32_t c = 0;
        first[0] = 0;
        for (int b = 1; b <= kHfLmax; ++b) {
            c = (c + cnt[b - 1]) << 1;
            first[b] = c;
        }
    }
    __syncthreads();
    uint32_t code = 0;
    if (l) {
        uint32_t before = 0;
        for (int s = 0; s < t; ++s) before += (len[s] == l) ? 1u : 0u;
        code = first[l] + before;
    }
    len_out[t] = (uint8_t)l;
    code_out[t] = code;
    hdr_len[t] = (uint8_t)l;
}

// Bits of each HF block (a warp per block): words[b] = ceil(bits / 32), also
// written to the stream's table, and the block's starting points: the bit
// offsets of its symbols 1024, 2048, 3072 (the bit count where the block is
// shorter), from the bits of its four quarters.
__global__ void __launch_bounds__(256) k_hf_count(const uint8_t* __restrict__ in, uint64_t n,
                                                  const uint8_t* __restrict__ len_g, uint32_t* __restrict__ words,
                                                  uint32_t* __restrict__ tab, uint16_t* __restrict__ sub_tab)
{
    __shared__ uint8_t len[256];
    len[threadIdx.x] = len_g[threadIdx.x];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nb = cr_nblocks(n);
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t b = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const uint64_t s0 = b * kHfBlock;
        const uint32_t cnt = (uint32_t)min((uint64_t)kHfBlock, n - s0);
        uint32_t qb[4] = {0u, 0u, 0u, 0u};  // bits of each quarter
        if (cnt == kHfBlock) {
            static_assert(kHfBlock == 4 * kHfSub && kHfSub == 16 * 64, "16-symbol vectors, 64 a quarter");
            const uint4* p = reinterpret_cast<const uint4*>(in + s0);
#pragma unroll
            for (uint32_t k = 0; k < kHfBlock / 16 / 32; ++k) {  // vector lane + 32 k is in quarter k / 2
                const uint4 q = __ldg(p + lane + 32 * k);
                const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
                uint32_t s = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) s += len[(wv[j] >> (8 * e)) & 0xffu];
                qb[k >> 1] += s;
            }
        } else {
            for (uint32_t i = lane; i < cnt; i += 32) {
                const uint32_t l = len[in[s0 + i]], qi = i / kHfSub;
                qb[0] += qi == 0 ? l : 0u;
                qb[1] += qi == 1 ? l : 0u;
                qb[2] += qi == 2 ? l : 0u;
                qb[3] += qi == 3 ? l : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) qb[j] = __reduce_add_sync(0xffffffffu, qb[j]);
        if (lane == 0) {
            const uint32_t bits = qb[0] + qb[1] + qb[2] + qb[3];
            const uint32_t wd = (bits + 31) / 32;
            words[b] = wd;
            tab[b] = wd;
            sub_tab[3 * b] = (uint16_t)qb[0];
            sub_tab[3 * b + 1] = (uint16_t)(qb[0] + qb[1]);
            sub_tab[3 * b + 2] = (uint16_t)(qb[0] + qb[1] + qb[2]);
            if (b == nb - 1 && (nb & 1)) sub_tab[3 * nb] = 0;  // the padding to 4 bytes
        }
    }
}

// Exclusive scan of cnt u32 values (one CTA of 1024 threads), each times
// scale, starting at base; returns the end through *total.  Each thread takes
// a contiguous run of ceil(cnt / threads) values: one pass for the run sums,
// one block scan of them, one pass writing the offsets.
__device__ __forceinline__ void cta_scan_u32(const uint32_t* in, uint32_t* out_or_null, uint64_t* out64_or_null,
                                             uint64_t cnt, uint64_t base, uint64_t* total, uint32_t scale)
{
    __shared__ uint64_t s_part[32];
    __shared__ uint64_t s_tot;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t per = (cnt + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = min(cnt, per * threadIdx.x), hi = min(cnt, lo + per);
    uint64_t mine = 0;
    for (uint64_t i = lo; i < hi; ++i) mine += (uint64_t)(in[i] & ~kCrRaw) * scale;
    uint64_t incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl += t;
    }
    if (lane == 31) s_part[warp] = incl;
    __syncthreads();
    uint64_t before = 0, tot = 0;
    for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) {
        before += (w < warp) ? s_part[w] : 0;
        tot += s_part[w];
    }
    uint64_t run = base + before + incl - mine;
    for (uint64_t i = lo; i < hi; ++i) {
        if (out_or_null) out_or_null[i] = (uint32_t)run;
        if (out64_or_null) out64_or_null[i] = run;
        run += (uint64_t)(in[i] & ~kCrRaw) * scale;
    }
    if (threadIdx.x == 0) s_tot = base + tot;
    __syncthreads();
    *total = s_tot;
    __syncthreads();
}

// Block word offsets and H; the stream's fixed header.
__global__ void __launch_bounds__(1024) k_cr_scan_words(const uint32_t* __restrict__ words, uint64_t n,
                                                         uint32_t* __restrict__ woff, uint64_t* __restrict__ hdr_ws,
                                                         uint8_t* __restrict__ out)
{
    const uint64_t nb = cr_nblocks(n);
    uint64_t tot = 0;
    cta_scan_u32(words, woff, nullptr, nb, 0, &tot, 1);
    if (threadIdx.x == 0) {
        const uint64_t H = 4 * tot;
        const uint32_t nc = (uint32_t)((H + kCrChunk - 1) / kCrChunk);
        hdr_ws[0] = H;
        reinterpret_cast<uint32_t*>(hdr_ws)[2] = nc;
        uint64_t* o64 = reinterpret_cast<uint64_t*>(out);
        uint32_t* o32 = reinterpret_cast<uint32_t*>(out);
        o64[0] = n;
        o32[2] = kHfBlock;
        o32[3] = (uint32_t)nb;
        o64[2] = H;
        o32[6] = kCrChunk;
        o32[7] = nc;
    }
}

// Pack each HF block's codes (a warp per block, 4 warps a CTA): the block's
// symbols staged in shared memory, each lane codes 128 consecutive symbols
// from the bit offset a warp scan gives it into shared-memory words (OR-ed,
// so the words a lane shares with its neighbours merge), then the words go
// out byte-swapped (the first bit is bit 7 of the first byte).
constexpr int kHfEncWarps = 2;
__global__ void __launch_bounds__(32 * kHfEncWarps) k_hf_encode(const uint8_t* __restrict__ in, uint64_t n,
                                                                const uint8_t* __restrict__ len_g,
                                                                const uint32_t* __restrict__ code_g,
                                                                const uint32_t* __restrict__ words,
                                                                const uint32_t* __restrict__ woff,
                                                                uint8_t* __restrict__ hf)
{
    __shared__ uint8_t len[256];
    __shared__ uint32_t code[256];
    __shared__ __align__(16) uint32_t s_sym[kHfEncWarps][kHfBlock / 4 + kHfBlock / 128];  // word w at w + w / 32
    __shared__ __align__(16) uint32_t s_bits[kHfEncWarps][kHfBlock * kHfLmax / 32];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        len[i] = len_g[i];
        code[i] = code_g[i];
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    uint32_t* symw = s_sym[wid];
    const uint8_t* sym = reinterpret_cast<const uint8_t*>(symw);
    uint32_t* bw = s_bits[wid];
    const uint64_t nb = cr_nblocks(n);
    const uint64_t warps = (uint64_t)gridDim.x * kHfEncWarps;
    for (uint64_t b = (uint64_t)blockIdx.x * kHfEncWarps + wid; b < nb; b += warps) {
        const uint64_t s0 = b * kHfBlock;
        const uint32_t cnt = (uint32_t)min((uint64_t)kHfBlock, n - s0);
        const uint32_t nw = words[b];
        if (cnt == kHfBlock) {
            for (uint32_t i = lane; i < kHfBlock / 16; i += 32) {
                const uint4 q = __ldg(reinterpret_cast<const uint4*>(in + s0) + i);
                const uint32_t w0 = 4 * i;  // the 4 words stay within one group of 32
                uint32_t* d = symw + w0 + w0 / 32;
                d[0] = q.x, d[1] = q.y, d[2] = q.z, d[3] = q.w;
            }
        } else {
            // a partial block (the last): symbols byte by byte into the skewed words
            for (uint32_t w = lane; w < kHfBlock / 4; w += 32) {
                uint32_t v = 0;
                for (uint32_t bb = 0; bb < 4; ++bb)
                    if (4 * w + bb < cnt) v |= (uint32_t)in[s0 + 4 * w + bb] << (8 * bb);
                symw[w + w / 32] = v;
            }
        }
        for (uint32_t i = lane; i < nw; i += 32) bw[i] = 0;
        __syncwarp();
        const uint32_t a = lane * (kHfBlock / 32);
        const uint32_t e = min(a + kHfBlock / 32, cnt);
        const bool whole = e == a + kHfBlock / 32;  // 128 symbols: read as words
        uint32_t mybits = 0;
        if (whole) {
#pragma unroll 4
            for (uint32_t q = a / 4; q < e / 4; ++q) {
                const uint32_t w4 = symw[q + q / 32];
                mybits += len[w4 & 0xffu] + len[(w4 >> 8) & 0xffu] + len[(w4 >> 16) & 0xffu] + len[w4 >> 24];
            }
        } else {
            for (uint32_t i = a; i < e; ++i) mybits += len[sym[i + 4 * (i / 128)]];
        }
        uint32_t incl = mybits;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += t;
        }
        const uint32_t pos = incl - mybits;
        uint32_t widx = pos >> 5;
        uint32_t nacc = pos & 31u;  // bits already taken in the first word (by earlier lanes)
        uint64_t acc = 0;
        // two codes at a time (at most 32 bits: with fewer than 32 pending the
        // 64-bit accumulator holds them), one word out whenever 32 are pending
        auto put = [&](uint32_t c2, uint32_t l2) {
            acc |= (uint64_t)c2 << (64 - nacc - l2);
            nacc += l2;
            if (nacc >= 32) {
                atomicOr(&bw[widx++], (uint32_t)(acc >> 32));
                acc <<= 32;
                nacc -= 32;
            }
        };
        if (whole) {
#pragma unroll 2
            for (uint32_t q = a / 4; q < e / 4; ++q) {
                const uint32_t w4 = symw[q + q / 32];
                const uint32_t s0 = w4 & 0xffu, s1 = (w4 >> 8) & 0xffu, s2 = (w4 >> 16) & 0xffu, s3 = w4 >> 24;
                const uint32_t l0 = len[s0], l1 = len[s1], l2 = len[s2], l3 = len[s3];
                const uint32_t c0 = code[s0], c1 = code[s1], c2 = code[s2], c3 = code[s3];
                put((c0 << l1) | c1, l0 + l1);
                put((c2 << l3) | c3, l2 + l3);
            }
        } else {
            for (uint32_t i = a; i < e; ++i) {
                const uint32_t sy = sym[i + 4 * (i / 128)];
                put(code[sy], len[sy]);
            }
        }
        if (nacc > 0 && mybits > 0) atomicOr(&bw[widx], (uint32_t)(acc >> 32));
        __syncwarp();
        uint32_t* dst = reinterpret_cast<uint32_t*>(hf) + woff[b];
        for (uint32_t i = lane; i < nw; i += 32) dst[i] = __byte_perm(bw[i], 0u, 0x0123);
        __syncwarp();
    }
}

// A CTA per 16 KiB chunk of the HF bytes: RRE4, TCMS8, RZE1 in shared
// memory; the payload (or the raw chunk) into the chunk's scratch slot.
// Shared-memory regions (bytes): the chunk; the RRE4 output r (= RZE1 level
// 0); the RZE1 levels 1..3; the RRE4 bitmap levels; the payload.
// RRE4 output: at most 64 + 512 bitmap bytes and 16384 kept bytes; every
// level buffer has room for its length rounded up to 64 plus one more span
// of zeros (span_flags reads whole 64-byte spans).
constexpr uint32_t kCrR = 16384 + 576 + 128;
constexpr uint32_t kCrZ1 = 2304;  // >= ceil(16960 / 8) rounded to 64, + 64
constexpr uint32_t kCrZ2 = 448;   // >= 265 -> 320, + 64
constexpr uint32_t kCrZ3 = 192;   // >= 34 -> 64, + 64
constexpr uint32_t kCrB0 = 640, kCrB1 = 128;
__host__ __device__ constexpr uint32_t r16(uint32_t b) { return (b + 15) / 16 * 16; }
constexpr uint32_t kOffIn = 0;
constexpr uint32_t kOffR = kOffIn + kCrChunk;
constexpr uint32_t kOffZ1 = kOffR + r16(kCrR);
constexpr uint32_t kOffZ2 = kOffZ1 + r16(kCrZ1);
constexpr uint32_t kOffZ3 = kOffZ2 + r16(kCrZ2);
constexpr uint32_t kOffB0 = kOffZ3 + r16(kCrZ3);
constexpr uint32_t kOffB1 = kOffB0 + r16(kCrB0);
constexpr uint32_t kOffPay = kOffB1 + r16(kCrB1);
constexpr uint32_t kCrSmem = kOffPay + kCrChunk + 64;
static_assert(kCrSmem <= 64 * 1024, "chunk shared memory");

__global__ void __launch_bounds__(kCrThreads) k_cr_lc_encode(const uint8_t* __restrict__ hf,
                                                             const uint64_t* __restrict__ hdr_ws,
                                                             uint8_t* __restrict__ slots, uint32_t* __restrict__ psize,
                                                             uint32_t* __restrict__ pm1)
{
    extern __shared__ __align__(16) unsigned char csm[];
    __shared__ uint32_t s_red[64];
    int parity = 0;
    const uint32_t t = threadIdx.x;
    uint8_t* cin = csm + kOffIn;
    uint8_t* r = csm + kOffR;
    uint8_t* z[4] = {r, csm + kOffZ1, csm + kOffZ2, csm + kOffZ3};
    uint8_t* b0 = csm + kOffB0;
    uint8_t* b1 = csm + kOffB1;
    uint8_t* pay = csm + kOffPay;
    const uint64_t H = hdr_ws[0];
    const uint32_t nc = reinterpret_cast<const uint32_t*>(hdr_ws)[2];
    for (uint32_t k = blockIdx.x; k < nc; k += gridDim.x) {
        const uint32_t m = (uint32_t)min((uint64_t)kCrChunk, H - (uint64_t)k * kCrChunk);  // a multiple of 4
        const uint32_t w = m / 4;
        const uint8_t* src = hf + (uint64_t)k * kCrChunk;
        for (uint32_t i = t; i < m / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(cin)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
        for (uint32_t i = m / 16 * 4 + t; i < w; i += blockDim.x)
            reinterpret_cast<uint32_t*>(cin)[i] = __ldg(reinterpret_cast<const uint32_t*>(src) + i);
        for (uint32_t i = t; i < kCrB0 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(b0)[i] = 0;
        for (uint32_t i = t; i < kCrB1 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(b1)[i] = 0;
        __syncthreads();
        // RRE4: word flags, 16 words a thread
        const uint32_t* cw = reinterpret_cast<const uint32_t*>(cin);
        uint32_t fm = 0;
        for (int j = 0; j < 16; ++j) {
            const uint32_t i = 16 * t + j;
            if (i < w && cw[i] != (i ? cw[i - 1] : 0u)) fm |= 1u << j;
        }
        const uint32_t L0 = (w + 7) / 8;
        if (2 * t < L0) b0[2 * t] = (uint8_t)fm;
        if (2 * t + 1 < L0) b0[2 * t + 1] = (uint8_t)(fm >> 8);
        uint32_t nkw = 0;
        const uint32_t kw_ex = cr_exscan((uint32_t)__popc(fm), s_red, parity, &nkw);  // barrier: b0 complete
        // RRE1 level of the bitmap when it is longer than 64 bytes (512 -> 64 at most)
        const bool two = L0 > 64;
        const uint32_t L1 = (L0 + 7) / 8;
        uint32_t m1a;
        if (two) {
            const uint32_t nk0 = level_bitmap(b0, L0, b1, false, s_red, parity);  // b0 zero padded to 576
            __syncthreads();
            for (uint32_t i = t; i < L1; i += blockDim.x) r[i] = b1[i];
            m1a = level_kept(b0, L0, b1, r, L1, s_red, parity);
            (void)nk0;
        } else {
            for (uint32_t i = t; i < L0; i += blockDim.x) r[i] = b0[i];
            m1a = L0;
        }
        // kept words after the bitmap section
        {
            uint32_t pos = m1a + 4 * kw_ex;
            uint32_t f = fm;
            while (f) {
                const int j = __ffs(f) - 1;
                f &= f - 1;
                const uint32_t v = cw[16 * t + j];
                r[pos] = (uint8_t)v;
                r[pos + 1] = (uint8_t)(v >> 8);
                r[pos + 2] = (uint8_t)(v >> 16);
                r[pos + 3] = (uint8_t)(v >> 24);
                pos += 4;
            }
        }
        const uint32_t m1 = m1a + 4 * nkw;
        __syncthreads();
        // TCMS8 on whole 8-byte words; zero pad to the next 64 bytes for the RZE1 spans
        for (uint32_t j = t; j < m1 / 8; j += blockDim.x) {
            const uint64_t v = reinterpret_cast<const uint64_t*>(r)[j];
            reinterpret_cast<uint64_t*>(r)[j] = (v << 1) ^ (uint64_t)((int64_t)v >> 63);
        }
        for (uint32_t i = m1 + t; i < (m1 + 63) / 64 * 64; i += blockDim.x) r[i] = 0;
        __syncthreads();
        // RZE1 levels
        const CrLevels T = cr_levels(m1);
        uint32_t total = T.L[T.R];
        for (int lv = 0; lv < T.R; ++lv) {
            // zero pad the next level to a multiple of 64 before it is read as spans
            const uint32_t Ln = T.L[lv + 1];
            for (uint32_t i = Ln + t; i < (Ln + 63) / 64 * 64 + 64; i += blockDim.x) z[lv + 1][i] = 0;
            __syncthreads();
            total += level_bitmap(z[lv], T.L[lv], z[lv + 1], true, s_red, parity);
            __syncthreads();
        }
        const bool raw = total > m;
        uint32_t plen = m;
        uint8_t* slot = slots + (uint64_t)k * kCrChunk;
        if (!raw) {
            for (uint32_t i = t; i < T.L[T.R]; i += blockDim.x) pay[i] = z[T.R][i];
            uint32_t off = T.L[T.R];
            for (int lv = T.R - 1; lv >= 0; --lv) off = level_kept(z[lv], T.L[lv], z[lv + 1], pay, off, s_red, parity);
            plen = off;
            const uint32_t pad = (plen + 15) / 16 * 16;
            for (uint32_t i = plen + t; i < pad; i += blockDim.x) pay[i] = 0;
            __syncthreads();
            for (uint32_t i = t; i < pad / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(slot)[i] = reinterpret_cast<const uint4*>(pay)[i];
            if (t == 0) {
                psize[k] = pad;
                pm1[k] = m1;
            }
        } else {
            for (uint32_t i = t; i < m / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(slot)[i] = reinterpret_cast<const uint4*>(cin)[i];
            for (uint32_t i = m / 16 * 4 + t; i < (m + 15) / 16 * 4; i += blockDim.x)
                reinterpret_cast<uint32_t*>(slot)[i] = (4 * i < m) ? reinterpret_cast<const uint32_t*>(cin)[i] : 0u;
            if (t == 0) {
                psize[k] = ((m + 15) / 16 * 16) | kCrRaw;
                pm1[k] = 0;
            }
        }
        __syncthreads();
    }
}

// Payload offsets; the chunk table and the stream length.
__global__ void __launch_bounds__(1024) k_cr_scan_payloads(const uint32_t* __restrict__ psize,
                                                            const uint32_t* __restrict__ pm1, uint64_t n,
                                                            const uint64_t* __restrict__ hdr_ws,
                                                            uint64_t* __restrict__ poff, uint8_t* __restrict__ out,
                                                            uint64_t* __restrict__ len)
{
    const uint64_t nb = cr_nblocks(n);
    const uint32_t nc = reinterpret_cast<const uint32_t*>(hdr_ws)[2];
    const uint64_t hb = cr_header_bytes(nb, nc);
    uint64_t tot = 0;
    cta_scan_u32(psize, nullptr, poff, nc, hb, &tot, 1);
    uint32_t* tab = reinterpret_cast<uint32_t*>(out + cr_tab_off(nb));
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
        tab[2 * i] = psize[i];
        tab[2 * i + 1] = pm1[i];
    }
    for (uint64_t i = cr_tab_off(nb) + 8 * (uint64_t)nc + threadIdx.x; i < hb; i += blockDim.x) out[i] = 0;
    if (threadIdx.x == 0) *len = tot;
}

__global__ void __launch_bounds__(256) k_cr_gather(const uint8_t* __restrict__ slots, const uint32_t* __restrict__ psize,
                                                   const uint64_t* __restrict__ poff,
                                                   const uint64_t* __restrict__ hdr_ws, uint8_t* __restrict__ out)
{
    const uint32_t nc = reinterpret_cast<const uint32_t*>(hdr_ws)[2];
    for (uint32_t k = blockIdx.x; k < nc; k += gridDim.x) {
        const uint32_t pad = psize[k] & ~kCrRaw;
        const uint4* s = reinterpret_cast<const uint4*>(slots + (uint64_t)k * kCrChunk);
        uint4* d = reinterpret_cast<uint4*>(out + poff[k]);
        for (uint32_t i = threadIdx.x; i < pad / 16; i += blockDim.x) d[i] = s[i];
    }
}

// ---------------------------------------------------------------------------
// Decode
// ---------------------------------------------------------------------------
// Offsets of the HF blocks and the payloads from the stream's tables; the
// header checked against n.
__global__ void __launch_bounds__(1024) k_cr_dec_scan(const uint8_t* __restrict__ in, uint64_t in_len, uint64_t n,
                                                       uint32_t* __restrict__ woff, uint64_t* __restrict__ poff,
                                                       uint64_t* __restrict__ hdr_ws, uint32_t* __restrict__ status)
{
    __shared__ int s_bad;
    const uint64_t* i64 = reinterpret_cast<const uint64_t*>(in);
    const uint32_t* i32 = reinterpret_cast<const uint32_t*>(in);
    const uint64_t nb = cr_nblocks(n);
    const uint64_t H = i64[2];
    const uint32_t nc = i32[7];
    if (threadIdx.x == 0) {
        int bad = i64[0] != n || i32[2] != kHfBlock || i32[3] != (uint32_t)nb || i32[6] != kCrChunk;
        bad = bad || H > cr_hmax(n) || (uint64_t)nc != (H + kCrChunk - 1) / kCrChunk || (H & 3);
        bad = bad || cr_header_bytes(nb, nc) > in_len;
        for (int v = 0; v < 256 && !bad; ++v) bad = in[32 + v] > kHfLmax;
        s_bad = bad;
    }
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) {
            set_status(status, HI_ECORRUPT);
            hdr_ws[0] = 0;
            reinterpret_cast<uint32_t*>(hdr_ws)[2] = 0;
            reinterpret_cast<uint32_t*>(hdr_ws)[3] = 1;  // decode nothing
        }
        return;
    }
    uint64_t wt = 0, pt = 0;
    cta_scan_u32(i32 + kCrHdr / 4, woff, nullptr, nb, 0, &wt, 1);
    // payload offsets: the sizes are every other word of the chunk table
    const uint32_t* tab = reinterpret_cast<const uint32_t*>(in + cr_tab_off(nb));
    {
        __shared__ uint64_t s_part[32];
        __shared__ uint64_t s_end;
        const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        const uint64_t per = ((uint64_t)nc + blockDim.x - 1) / blockDim.x;
        const uint64_t lo = min((uint64_t)nc, per * threadIdx.x), hi = min((uint64_t)nc, lo + per);
        uint64_t mine = 0;
        for (uint64_t i = lo; i < hi; ++i) mine += tab[2 * i] & ~kCrRaw;
        uint64_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t tt = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += tt;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        uint64_t before = 0, tot = 0;
        for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) {
            before += (w < warp) ? s_part[w] : 0;
            tot += s_part[w];
        }
        const uint64_t hb = cr_header_bytes(nb, nc);
        uint64_t run = hb + before + incl - mine;
        for (uint64_t i = lo; i < hi; ++i) {
            poff[i] = run;
            run += tab[2 * i] & ~kCrRaw;
        }
        if (threadIdx.x == 0) s_end = hb + tot;
        __syncthreads();
        pt = s_end;
    }
    if (threadIdx.x == 0) {
        const bool bad = 4 * wt != H || pt > in_len;
        if (bad) set_status(status, HI_ECORRUPT);
        hdr_ws[0] = H;
        reinterpret_cast<uint32_t*>(hdr_ws)[2] = bad ? 0u : nc;
        reinterpret_cast<uint32_t*>(hdr_ws)[3] = bad ? 1u : 0u;
    }
}

// Level lv of a chunk from its bitmap (level lv + 1) and the kept bytes at
// p[q..): zero elimination puts 0 at unflagged positions, repeat elimination
// the previous byte (the kept byte of rank popcount(bitmap[0..i]) - 1, or 0).
// Returns q advanced past the kept bytes; *bad set when they run past avail.
__device__ __forceinline__ uint32_t level_expand(const uint8_t* bm, uint32_t L, const uint8_t* p, uint32_t q,
                                                 uint32_t avail, bool zero, uint8_t* dst, uint32_t* s_red, int& parity,
                                                 bool* bad)
{
    for (uint32_t a0 = 0; a0 < L; a0 += 64 * blockDim.x) {
        const uint32_t a = a0 + 64 * threadIdx.x;
        uint64_t f = 0;
        if (a < L) {
            const uint2 b = reinterpret_cast<const uint2*>(bm)[a / 64];
            f = (uint64_t)b.x | ((uint64_t)b.y << 32);
            const uint32_t valid = L - a;
            if (valid < 64) f &= (1ull << valid) - 1ull;
        }
        uint32_t tot;
        const uint32_t ex = cr_exscan((uint32_t)__popcll(f), s_red, parity, &tot);
        if (q + tot > avail) *bad = true;
        if (a < L && q + tot <= avail) {
            uint32_t rel = ex;  // kept bytes of this level before this span
            const uint32_t e = min(64u, L - a);
            for (uint32_t i = 0; i < e; ++i) {
                uint8_t v;
                if ((f >> i) & 1) {
                    v = p[q + rel++];
                } else if (zero) {
                    v = 0;
                } else {
                    v = rel > 0 ? p[q + rel - 1] : 0;  // repeat: the last kept byte so far (0 before any)
                }
                dst[a + i] = v;
            }
        }
        q += tot;
    }
    return q;
}

__global__ void __launch_bounds__(kCrThreads) k_cr_lc_decode(const uint8_t* __restrict__ in,
                                                             const uint64_t* __restrict__ poff, uint64_t n,
                                                             const uint64_t* __restrict__ hdr_ws, uint8_t* __restrict__ hf,
                                                             uint32_t* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char csm[];
    __shared__ uint32_t s_red[64];
    __shared__ int s_bad;
    int parity = 0;
    const uint32_t t = threadIdx.x;
    uint8_t* pin = csm + kOffIn;  // the payload (at most a chunk)
    uint8_t* z[4] = {csm + kOffR, csm + kOffZ1, csm + kOffZ2, csm + kOffZ3};
    uint8_t* b0 = csm + kOffB0;
    const uint64_t H = hdr_ws[0];
    const uint32_t nc = reinterpret_cast<const uint32_t*>(hdr_ws)[2];
    const uint64_t nb = cr_nblocks(n);
    const uint32_t* tab = reinterpret_cast<const uint32_t*>(in + cr_tab_off(nb));
    for (uint32_t k = blockIdx.x; k < nc; k += gridDim.x) {
        const uint32_t m = (uint32_t)min((uint64_t)kCrChunk, H - (uint64_t)k * kCrChunk);
        const uint32_t sz = tab[2 * k], m1 = tab[2 * k + 1];
        const uint32_t pad = sz & ~kCrRaw;
        const uint8_t* p = in + poff[k];
        uint8_t* dst = hf + (uint64_t)k * kCrChunk;
        if (sz & kCrRaw) {
            if (pad < m || pad > kCrChunk) {
                if (t == 0) set_status(status, HI_ECORRUPT);
                continue;
            }
            for (uint32_t i = t; i < m / 4; i += blockDim.x)
                reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(p)[i];
            continue;
        }
        if (pad > kCrChunk || m1 > kCrR - 64 || m1 == 0) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            continue;
        }
        for (uint32_t i = t; i < pad / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(pin)[i] = reinterpret_cast<const uint4*>(p)[i];
        if (t == 0) s_bad = 0;
        __syncthreads();
        bool bad = false;
        // RZE1 levels, top down
        const CrLevels T = cr_levels(m1);
        if (T.L[T.R] > pad) bad = true;
        for (uint32_t i = t; i < T.L[T.R] && !bad; i += blockDim.x) z[T.R][i] = pin[i];
        for (uint32_t i = T.L[T.R] + t; i < (T.L[T.R] + 63) / 64 * 64 + 64; i += blockDim.x) z[T.R][i] = 0;
        __syncthreads();
        uint32_t q = T.L[T.R];
        for (int lv = T.R - 1; lv >= 0 && !bad; --lv) {
            q = level_expand(z[lv + 1], T.L[lv], pin, q, pad, true, z[lv], s_red, parity, &bad);
            __syncthreads();
        }
        if (bad) s_bad = 1;
        __syncthreads();
        if (s_bad) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            continue;
        }
        uint8_t* r = z[0];
        // TCMS8 inverse
        for (uint32_t j = t; j < m1 / 8; j += blockDim.x) {
            const uint64_t u = reinterpret_cast<const uint64_t*>(r)[j];
            reinterpret_cast<uint64_t*>(r)[j] = (u >> 1) ^ (0ull - (u & 1ull));
        }
        __syncthreads();
        // RRE4 inverse: the bitmap (through its RRE1 level when longer than 64 bytes), then the words
        const uint32_t w = m / 4, L0 = (w + 7) / 8;
        uint32_t m1a;
        if (L0 > 64) {
            const uint32_t L1 = (L0 + 7) / 8;
            for (uint32_t i = t; i < kCrB1; i += blockDim.x) z[3][i] = i < L1 ? r[i] : 0;  // level 1 (z3 is free now)
            __syncthreads();
            m1a = level_expand(z[3], L0, r, L1, m1, false, b0, s_red, parity, &bad);
        } else {
            for (uint32_t i = t; i < L0; i += blockDim.x) b0[i] = r[i];
            m1a = L0;
        }
        for (uint32_t i = L0 + t; i < kCrB0; i += blockDim.x) b0[i] = 0;
        __syncthreads();
        const uint32_t fm = (16 * t < w) ? ((uint32_t)b0[2 * t] | ((uint32_t)b0[2 * t + 1] << 8)) &
                                               ((16 * t + 16 <= w) ? 0xffffu : ((1u << (w - 16 * t)) - 1u))
                                         : 0u;
        uint32_t nkw = 0;
        const uint32_t ex = cr_exscan((uint32_t)__popc(fm), s_red, parity, &nkw);
        if (m1a + 4 * nkw > m1) bad = true;
        if (bad) s_bad = 1;
        __syncthreads();
        if (s_bad) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            continue;
        }
        uint32_t rank = ex;
        for (int j = 0; j < 16; ++j) {
            const uint32_t i = 16 * t + j;
            if (i >= w) break;
            if ((fm >> j) & 1) ++rank;
            uint32_t v = 0;
            if (rank > 0) {
                const uint8_t* kp = r + m1a + 4 * (rank - 1);
                v = (uint32_t)kp[0] | ((uint32_t)kp[1] << 8) | ((uint32_t)kp[2] << 16) | ((uint32_t)kp[3] << 24);
            }
            reinterpret_cast<uint32_t*>(dst)[i] = v;
        }
        __syncthreads();
    }
}

// A thread per HF block: canonical decoding through a 12-bit table (codes
// up to 12 bits in one lookup); a longer code's length comes from comparing
// the next 16 bits against the end of each longer length's code range
// (canonical codes of one length are consecutive), branch-free.  The next
// stream word is loaded one refill ahead (its latency hides behind a dozen
// symbols) and the output leaves in 16-byte stores.
constexpr int kHfDecThreads = 256;
__global__ void __launch_bounds__(kHfDecThreads) k_hf_decode(const uint8_t* __restrict__ in,
                                                             const uint8_t* __restrict__ hf,
                                                             const uint32_t* __restrict__ woff, uint64_t n,
                                                             const uint64_t* __restrict__ hdr_ws,
                                                             uint8_t* __restrict__ out, uint32_t* __restrict__ status)
{
    __shared__ uint16_t lut[1 << kHfLut];  // symbol | length << 8, 0 = longer code
    __shared__ uint8_t len[256], sorted[256];
    __shared__ uint32_t cnt[kHfLmax + 1], first[kHfLmax + 1], offs[kHfLmax + 1], lim[kHfLmax + 1];
    if (reinterpret_cast<const uint32_t*>(hdr_ws)[3]) return;  // the header did not check out
    const int t = threadIdx.x;
    for (int i = t; i < 256; i += blockDim.x) len[i] = in[32 + i];
    for (int i = t; i < (1 << kHfLut); i += blockDim.x) lut[i] = 0;
    if (t <= kHfLmax) cnt[t] = 0;
    __syncthreads();
    for (int v = t; v < 256; v += blockDim.x)
        if (len[v]) atomicAdd(&cnt[len[v]], 1u);
    __syncthreads();
    if (t == 0) {
        uint32_t c = 0, ns = 0, prev = 0;
        for (int l = 1; l <= kHfLmax; ++l) {
            c = (c + prev) << 1;
            first[l] = c;
            offs[l] = ns;
            ns += cnt[l];
            prev = cnt[l];
            lim[l] = (c + cnt[l]) << (kHfLmax - l);  // 16-bit windows below this start a code of length <= l
        }
    }
    __syncthreads();
    for (int v = t; v < 256; v += blockDim.x) {  // (length, symbol) order; table entries of the short codes
        const int l = len[v];
        if (l == 0) continue;
        uint32_t rank = 0;
        for (int s = 0; s < v; ++s) rank += (len[s] == l) ? 1u : 0u;
        sorted[offs[l] + rank] = (uint8_t)v;
        if (l > kHfLut) continue;
        const uint32_t base = (first[l] + rank) << (kHfLut - l);
        for (uint32_t j = 0; j < (1u << (kHfLut - l)); ++j) lut[base + j] = (uint16_t)(v | (l << 8));
    }
    __syncthreads();
    // lengths 13..16: a window w16 of the next 16 bits starts a code of length
    // 13 + (w16 >= lim[13]) + (w16 >= lim[14]) + (w16 >= lim[15]); valid when w16 < lim[16]
    const uint32_t lim13 = lim[13], lim14 = lim[14], lim15 = lim[15], lim16 = lim[16];
    const uint64_t nb = cr_nblocks(n);
    const uint32_t* words = reinterpret_cast<const uint32_t*>(in + kCrHdr);
    const uint16_t* subs = reinterpret_cast<const uint16_t*>(in + kCrHdr + 4 * nb);
    // a thread per quarter of a block: from its starting point in the table,
    // its (up to) 1024 symbols; it must end where the next starting point is
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + t; u < 4 * nb; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = u >> 2;
        const uint32_t j = (uint32_t)(u & 3u);
        const uint64_t s0 = b * kHfBlock;
        const uint32_t cnt_blk = (uint32_t)min((uint64_t)kHfBlock, n - s0);
        const uint32_t i0 = j * kHfSub;
        if (i0 >= cnt_blk) continue;
        const uint32_t cntb = min(kHfSub, cnt_blk - i0);
        const uint64_t base = s0 + i0;
        const uint32_t nw = words[b];
        const uint32_t start = j ? subs[3 * b + j - 1] : 0u;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(hf) + woff[b];
        auto word = [&](uint32_t k) -> uint32_t { return k < nw ? __byte_perm(__ldg(src + k), 0u, 0x0123) : 0u; };
        const uint32_t k0 = start >> 5, sh = start & 31u;
        uint64_t buf = (((uint64_t)word(k0) << 32) | word(k0 + 1)) << sh;  // upcoming bits, MSB first
        uint32_t have = 64 - sh;
        // the next three words, loaded three refills (some 40 symbols) before they are needed
        uint32_t pre0 = word(k0 + 2), pre1 = word(k0 + 3), pre2 = word(k0 + 4);
        uint32_t wi = k0 + 5;  // next word to load
        bool bad = start > 32u * nw;
        uint32_t o0 = 0, o1 = 0, o2 = 0, cur = 0;
        for (uint32_t i = 0; i < cntb && !bad; ++i) {
            if (have <= 32) {
                buf |= (uint64_t)pre0 << (32 - have);
                have += 32;
                pre0 = pre1;
                pre1 = pre2;
                pre2 = word(wi);
                ++wi;
            }
            const uint32_t e = lut[(uint32_t)(buf >> (64 - kHfLut))];
            uint32_t sym, l;
            if (e) {
                sym = e & 0xffu;
                l = e >> 8;
            } else {
                const uint32_t w16 = (uint32_t)(buf >> (64 - kHfLmax));
                l = 13 + (w16 >= lim13 ? 1u : 0u) + (w16 >= lim14 ? 1u : 0u) + (w16 >= lim15 ? 1u : 0u);
                const uint32_t c = w16 >> (kHfLmax - l);
                const uint32_t k = c - first[l];
                if (w16 >= lim16 || k >= cnt[l]) {
                    bad = true;
                    break;
                }
                sym = sorted[offs[l] + k];
            }
            buf <<= l;
            have -= l;
            cur |= sym << (8 * (i & 3));
            if ((i & 3) == 3) {
                if ((i & 15) == 15) {
                    *reinterpret_cast<uint4*>(out + base + i - 15) = make_uint4(o0, o1, o2, cur);
                } else {
                    o0 = o1;
                    o1 = o2;
                    o2 = cur;
                }
                cur = 0;
            }
        }
        if (!bad) {
            // the symbols after the last 16-byte store: up to three words in o*, then cur
            const uint32_t done = cntb & ~15u, rem = cntb - done;
            const uint32_t wds = rem / 4;
            const uint32_t ow[3] = {wds == 3 ? o0 : (wds == 2 ? o1 : o2), wds == 3 ? o1 : o2, o2};
            for (uint32_t k = 0; k < wds; ++k)
                *reinterpret_cast<uint32_t*>(out + base + done + 4 * k) = ow[k];
            for (uint32_t k = done + 4 * wds; k < cntb; ++k) out[base + k] = (uint8_t)(cur >> (8 * (k & 3)));
            // the bit position reached (wi - 3 words have entered buf): the next starting point,
            // and within the block's words
            const uint64_t pos = 32ull * (wi - 3) - have;
            if (pos > 32ull * nw || (j < 3 && pos != subs[3 * b + j])) bad = true;
        }
        if (bad) set_status(status, HI_ECORRUPT);
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
size_t cr_ws_bytes(uint64_t n) { return (size_t)cr_ws(n).total; }
uint64_t cr_stream_bound(uint64_t n) { return cr_header_bytes(cr_nblocks(n), cr_ncmax(n)) + cr_hmax(n) + 16 * cr_ncmax(n) + 16; }

static int cr_grid(uint64_t units, int per_sm, int num_sms)
{
    const uint64_t g = (uint64_t)per_sm * (uint64_t)num_sms;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(units, g));
}

cudaError_t launch_cr_encode(const uint8_t* in, uint64_t n, uint8_t* out, uint64_t* len, void* ws_v, int num_sms,
                             cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_cr_lc_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, kCrSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    uint8_t* ws = static_cast<uint8_t*>(ws_v);
    const CrWs L = cr_ws(n);
    const uint64_t nb = cr_nblocks(n), ncm = cr_ncmax(n);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
    uint8_t* lens = ws + L.book;
    uint32_t* codes = reinterpret_cast<uint32_t*>(ws + L.book + 256);
    uint64_t* hdr = reinterpret_cast<uint64_t*>(ws + L.hdr);
    uint32_t* words = reinterpret_cast<uint32_t*>(ws + L.words);
    uint32_t* woff = reinterpret_cast<uint32_t*>(ws + L.woff);
    uint32_t* psize = reinterpret_cast<uint32_t*>(ws + L.psize);
    uint32_t* pm1 = reinterpret_cast<uint32_t*>(ws + L.pm1);
    uint64_t* poff = reinterpret_cast<uint64_t*>(ws + L.poff);
    uint8_t* hf = ws + L.hf;
    uint8_t* slots = ws + L.slots;
    cudaError_t e = cudaMemsetAsync(hist, 0, 1024, st);
    if (e != cudaSuccess) return e;
    k_cr_hist<<<cr_grid((n / 16 + 255) / 256, 8, num_sms), 256, 0, st>>>(in, n, hist);
    k_cr_codebook<<<1, 32 * kBookWarps, 0, st>>>(hist, lens, codes, out + 32);
    k_hf_count<<<cr_grid((nb + 7) / 8, 8, num_sms), 256, 0, st>>>(
        in, n, lens, words, reinterpret_cast<uint32_t*>(out + kCrHdr), reinterpret_cast<uint16_t*>(out + kCrHdr + 4 * nb));
    k_cr_scan_words<<<1, 1024, 0, st>>>(words, n, woff, hdr, out);
    k_hf_encode<<<cr_grid((nb + kHfEncWarps - 1) / kHfEncWarps, 8, num_sms), 32 * kHfEncWarps, 0, st>>>(
        in, n, lens, codes, words, woff, hf);
    k_cr_lc_encode<<<cr_grid(ncm, 3, num_sms), kCrThreads, kCrSmem, st>>>(hf, hdr, slots, psize, pm1);
    k_cr_scan_payloads<<<1, 1024, 0, st>>>(psize, pm1, n, hdr, poff, out, len);
    k_cr_gather<<<cr_grid(ncm, 4, num_sms), 256, 0, st>>>(slots, psize, poff, hdr, out);
    return cudaGetLastError();
}

cudaError_t launch_cr_decode(const uint8_t* in, uint64_t in_len, uint64_t n, uint8_t* out, uint32_t* status,
                             void* ws_v, int num_sms, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_cr_lc_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, kCrSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    uint8_t* ws = static_cast<uint8_t*>(ws_v);
    const CrWs L = cr_ws(n);
    const uint64_t nb = cr_nblocks(n), ncm = cr_ncmax(n);
    uint64_t* hdr = reinterpret_cast<uint64_t*>(ws + L.hdr);
    uint32_t* woff = reinterpret_cast<uint32_t*>(ws + L.woff);
    uint64_t* poff = reinterpret_cast<uint64_t*>(ws + L.poff);
    uint8_t* hf = ws + L.hf;
    k_cr_dec_scan<<<1, 1024, 0, st>>>(in, in_len, n, woff, poff, hdr, status);
    k_cr_lc_decode<<<cr_grid(ncm, 3, num_sms), kCrThreads, kCrSmem, st>>>(in, poff, n, hdr, hf, status);
    k_hf_decode<<<cr_grid((4 * nb + kHfDecThreads - 1) / kHfDecThreads, 8, num_sms), kHfDecThreads, 0, st>>>(
        in, hf, woff, n, hdr, out, status);
    return cudaGetLastError();
}

}  // namespace hi
