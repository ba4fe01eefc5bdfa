// hi_tp.cu -- the throughput-mode lossless pipeline TCMS1-BIT1-RRE1 of
// cuSZ-Hi (arXiv 2507.11165, Sec. 5.2.3) over a byte sequence (the
// reordered quantization codes), and its inverse.  The paper names the
// stages; the container is this library's reading:
//   stream  = u64 n | u32 chunk | u32 nchunks | u32 size[nchunks] | zero pad
//             to 16 bytes | payloads (each padded to 16 bytes)
//   size[k] = padded payload bytes, bit 31 = chunk stored raw
//   TCMS1   t = (b << 1) ^ (b >> 7), b read as a signed int8
//   BIT1    t zero-padded to m' (m rounded up to 64); plane p = bit 7 - p of
//           every element, element 8 j + b at bit b of the plane's byte j
//   RRE1    bitmap bit i = (v[i] != v[i - 1]), v[-1] = 0, LSB first; kept =
//           the bytes whose bit is set; applied to its own bitmap until a
//           level has at most 64 bytes, which is stored as is
//   payload = top level | kept of the levels below, top down; raw (m bytes)
//             when that would be longer than m.
// Encoding: a CTA per chunk, a thread per 64 bytes of it -- the transform
// four bytes at a time, an 8x8 bit transpose per 8 elements for the bit
// planes, changed-byte flags from byte-exact compares for the bitmaps, kept
// bytes placed by a block prefix sum into the payload staged in shared
// memory -- into a scratch slot per chunk; a scan of the sizes; a gather of
// the payloads.  Decoding: the scan, then a CTA per chunk expanding the
// levels top down (the byte at i is the kept byte of rank popcount(bitmap
// [0..i])) and transposing the bit planes back.
#include "hi_internal.h"
#include "hi_device.cuh"

namespace hi {

constexpr uint32_t kTpChunk = 16384;
constexpr uint32_t kTpRaw = 0x80000000u;
constexpr uint32_t kTpSlot = kTpChunk + 64;  // scratch bytes per chunk (16-byte multiple)
constexpr int kTpThreads = 256;
constexpr int kTpMaxLevels = 6;

__host__ __device__ constexpr uint64_t tp_header_bytes(uint64_t nchunks) { return (16 + 4 * nchunks + 15) / 16 * 16; }

struct TpLevels {
    uint32_t L[kTpMaxLevels];
    int R;  // top level
};

__device__ __forceinline__ TpLevels tp_levels(uint32_t m)
{
    TpLevels T;
    T.L[0] = (m + 63) / 64 * 64;
    T.R = 0;
    while (T.L[T.R] > 64) {
        T.L[T.R + 1] = (T.L[T.R] + 7) / 8;
        ++T.R;
    }
    return T;
}

// Offsets (bytes) of the level buffers in shared memory: level 0 holds m'
// <= kTpChunk bytes, level r > 0 at most kTpChunk / 8^r; each with 64 bytes
// of slack for whole-word bitmap writes.
__host__ __device__ constexpr uint32_t tp_level_off(int r)
{
    uint32_t o = 0, len = kTpChunk;
    for (int k = 0; k < r; ++k) {
        o += (len + 64 + 15) / 16 * 16;
        len /= 8;
    }
    return o;
}
constexpr uint32_t kTpLevelBytes = tp_level_off(kTpMaxLevels);
static_assert(kTpLevelBytes < 20 * 1024, "level buffers");

// Four bytes at a time: TCMS1 on each byte of w, and its inverse.
__device__ __forceinline__ uint32_t tcms1_4(uint32_t w)
{
    return ((w << 1) & 0xfefefefeu) ^ (((w >> 7) & 0x01010101u) * 0xffu);
}
__device__ __forceinline__ uint32_t tcms1_inv_4(uint32_t t)
{
    return ((t >> 1) & 0x7f7f7f7fu) ^ ((t & 0x01010101u) * 0xffu);
}

// 8x8 bit transpose (Hacker's Delight, transpose8 with 64-bit delta swaps):
// bit 8 i + j of x goes to bit 8 j + i.  With byte i = element i, byte j of
// the result holds bit j of every element, element i at bit i.
__device__ __forceinline__ uint64_t transpose8(uint64_t x)
{
    uint64_t t = (x ^ (x >> 7)) & 0x00aa00aa00aa00aaull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000cccc0000ccccull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000f0f0f0f0ull;
    return x ^ t ^ (t << 28);
}

// Bit k (k < 4) set when byte k of w differs from the byte before it (prev:
// the word before w).  Nonzero bytes of the xor are found exactly (no carry
// between bytes) and their top bits gathered by one multiply.
__device__ __forceinline__ uint32_t diff_flags4(uint32_t w, uint32_t prev)
{
    const uint32_t d = w ^ __funnelshift_l(prev, w, 8);
    const uint32_t nz = (((d & 0x7f7f7f7fu) + 0x7f7f7f7fu) | d) & 0x80808080u;
    return (((nz >> 7) * 0x00204081u) >> 21) & 0xfu;
}

// Flags of positions a .. a + 4 W - 1 of level v (bit i: v[a + i] differs
// from its predecessor, v[-1] = 0), cleared at and past L.  a is a multiple
// of 4 W.
template <int W>
__device__ __forceinline__ uint64_t range_flags(const uint8_t* v, uint32_t a, uint32_t L)
{
    uint32_t prev = a ? (uint32_t)v[a - 1] << 24 : 0u;
    uint64_t f = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const uint32_t w = reinterpret_cast<const uint32_t*>(v + a)[k];
        f |= (uint64_t)diff_flags4(w, prev) << (4 * k);
        prev = w;
    }
    if (a + 4 * W > L) {
        const uint32_t valid = L > a ? L - a : 0u;
        f &= valid >= 64 ? ~0ull : ((1ull << valid) - 1ull);
    }
    return f;
}

// Exclusive prefix over the block of one count per thread; *total = the sum.
// s_red holds two arrays of a word per warp, used by alternate calls
// (parity): a call writes the array that the previous call did not read,
// and every thread has finished reading the one before that when it
// reaches the previous call's barrier, so one barrier per call suffices.
__device__ __forceinline__ uint32_t block_exscan(uint32_t c, uint32_t* s_red, int& parity, uint32_t* total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t* part = s_red + (parity ? kTpThreads / 32 : 0);
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

// Level r of a chunk: a thread covers 64 positions at level 0, 8 above.
__device__ __forceinline__ uint32_t level_span(int r) { return r == 0 ? 64u : 8u; }

// Bitmap bits of level r's positions [a, a + span) read from the level
// above (bitmap buffer bm), cleared at and past L.
__device__ __forceinline__ uint64_t level_bits(const uint8_t* bm, int r, uint32_t t, uint32_t L)
{
    const uint32_t a = level_span(r) * t;
    uint64_t f = (r == 0) ? reinterpret_cast<const uint64_t*>(bm)[t] : (uint64_t)bm[t];
    if (a + level_span(r) > L) {
        const uint32_t valid = L > a ? L - a : 0u;
        f &= valid >= 64 ? ~0ull : ((1ull << valid) - 1ull);
    }
    return f;
}

__global__ void __launch_bounds__(kTpThreads) k_tp_encode_chunks(const uint8_t* __restrict__ in, uint64_t n,
                                                                 uint8_t* __restrict__ slots,
                                                                 uint32_t* __restrict__ sizes, uint32_t nchunks)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ uint32_t s_red[2 * (kTpThreads / 32)];
    int parity = 0;
    const uint32_t t = threadIdx.x;
    uint8_t* sin = tsm + kTpLevelBytes;  // the chunk's input, then its payload
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint8_t* s = in + (uint64_t)k * kTpChunk;
        const uint32_t m = (uint32_t)min((uint64_t)kTpChunk, n - (uint64_t)k * kTpChunk);
        const TpLevels T = tp_levels(m);
        const uint32_t mp = T.L[0];
        if ((reinterpret_cast<uintptr_t>(s) & 15u) == 0) {
            for (uint32_t i = t; i < m / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(sin)[i] = __ldg(reinterpret_cast<const uint4*>(s) + i);
            for (uint32_t i = m / 16 * 16 + t; i < m; i += blockDim.x) sin[i] = s[i];
        } else {
            for (uint32_t i = t; i < m; i += blockDim.x) sin[i] = s[i];
        }
        for (uint32_t i = m + t; i < mp; i += blockDim.x) sin[i] = 0;  // TCMS1(0) = 0: the zero padding
        __syncthreads();
        // TCMS1 + BIT1: elements 64 t .. 64 t + 63 -> bytes 8 t .. 8 t + 7 of each plane
        uint8_t* u = tsm + tp_level_off(0);
        const uint32_t pl = mp / 8;
        if (64 * t < mp) {
            uint64_t tr[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const uint2 w = reinterpret_cast<const uint2*>(sin + 64 * t)[g];
                tr[g] = transpose8((uint64_t)tcms1_4(w.x) | ((uint64_t)tcms1_4(w.y) << 32));
            }
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const int b = 7 - p;  // byte of each transposed group holding plane p
                uint32_t h[8];
#pragma unroll
                for (int g = 0; g < 8; ++g) h[g] = (uint32_t)(tr[g] >> (b >= 4 ? 32 : 0));
                const uint32_t sel = (uint32_t)(b & 3) | ((uint32_t)(4 + (b & 3)) << 4);
                const uint32_t lo = __byte_perm(__byte_perm(h[0], h[1], sel), __byte_perm(h[2], h[3], sel), 0x5410);
                const uint32_t hi = __byte_perm(__byte_perm(h[4], h[5], sel), __byte_perm(h[6], h[7], sel), 0x5410);
                reinterpret_cast<uint2*>(u + p * pl)[t] = make_uint2(lo, hi);
            }
        }
        __syncthreads();
        // RRE1 bitmaps, level by level
        uint32_t total = T.L[T.R];
        for (int r = 0; r < T.R; ++r) {
            const uint8_t* v = tsm + tp_level_off(r);
            uint8_t* bm = tsm + tp_level_off(r + 1);
            const uint32_t span = level_span(r);
            uint64_t f = 0;
            if (span * t < T.L[r]) {
                if (r == 0) {
                    f = range_flags<16>(v, 64 * t, T.L[r]);
                    reinterpret_cast<uint64_t*>(bm)[t] = f;
                } else {
                    f = range_flags<2>(v, 8 * t, T.L[r]);
                    bm[t] = (uint8_t)f;
                }
            }
            uint32_t c_tot;
            block_exscan((uint32_t)__popcll(f), s_red, parity, &c_tot);
            total += c_tot;
        }
        uint8_t* slot = slots + (uint64_t)k * kTpSlot;
        const bool raw = total > m;
        uint32_t len = m;
        if (!raw) {
            // payload in sin: top level, then the kept bytes of each level below it
            const uint8_t* top = tsm + tp_level_off(T.R);
            for (uint32_t i = t; i < T.L[T.R]; i += blockDim.x) sin[i] = top[i];
            uint32_t off = T.L[T.R];
            for (int r = T.R - 1; r >= 0; --r) {
                const uint8_t* v = tsm + tp_level_off(r);
                const uint32_t a = level_span(r) * t;
                uint64_t f = (a < T.L[r]) ? level_bits(tsm + tp_level_off(r + 1), r, t, T.L[r]) : 0ull;
                uint32_t c_tot;
                uint32_t pos = off + block_exscan((uint32_t)__popcll(f), s_red, parity, &c_tot);
                while (f) {
                    const int i = __ffsll((long long)f) - 1;
                    f &= f - 1;
                    sin[pos++] = v[a + i];
                }
                off += c_tot;
            }
            len = off;
        }
        const uint32_t pad = (len + 15) / 16 * 16;
        for (uint32_t i = len + t; i < pad; i += blockDim.x) sin[i] = 0;
        __syncthreads();
        for (uint32_t i = t; i < pad / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(slot)[i] = reinterpret_cast<const uint4*>(sin)[i];
        if (t == 0) sizes[k] = pad | (raw ? kTpRaw : 0u);
        __syncthreads();  // shared buffers are reused by the next chunk
    }
}

// Exclusive scan of the padded sizes (one CTA): offsets[k] = header +
// sum of sizes before k; with out != nullptr also writes the stream header
// and size table, and the stream length to *len.
__global__ void __launch_bounds__(1024) k_tp_scan(const uint32_t* __restrict__ sizes, uint32_t nchunks, uint64_t n,
                                                  uint64_t* __restrict__ offsets, uint8_t* __restrict__ out,
                                                  uint64_t* __restrict__ len)
{
    __shared__ uint64_t s_part[32];
    __shared__ uint64_t s_base;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = tp_header_bytes(nchunks);
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nchunks; c0 += blockDim.x) {
        const uint32_t k = c0 + threadIdx.x;
        const uint32_t raw = k < nchunks ? sizes[k] : 0u;
        const uint64_t v = raw & ~kTpRaw;
        uint64_t incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += t;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        uint64_t before = s_base;
        for (uint32_t w = 0; w < warp; ++w) before += s_part[w];
        if (k < nchunks) {
            offsets[k] = before + incl - v;
            if (out) reinterpret_cast<uint32_t*>(out + 16)[k] = raw;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            uint64_t t = 0;
            for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += s_part[w];
            s_base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && out) {
        reinterpret_cast<uint64_t*>(out)[0] = n;
        reinterpret_cast<uint32_t*>(out)[2] = kTpChunk;
        reinterpret_cast<uint32_t*>(out)[3] = nchunks;
        for (uint64_t b = 16 + 4 * (uint64_t)nchunks; b < tp_header_bytes(nchunks); ++b) out[b] = 0;
        *len = s_base;
    }
}

__global__ void __launch_bounds__(256) k_tp_gather(const uint8_t* __restrict__ slots,
                                                   const uint32_t* __restrict__ sizes,
                                                   const uint64_t* __restrict__ offsets, uint32_t nchunks,
                                                   uint8_t* __restrict__ out)
{
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint32_t pad = sizes[k] & ~kTpRaw;
        const uint4* src = reinterpret_cast<const uint4*>(slots + (uint64_t)k * kTpSlot);
        uint4* dst = reinterpret_cast<uint4*>(out + offsets[k]);
        for (uint32_t i = threadIdx.x; i < pad / 16; i += blockDim.x) dst[i] = src[i];
    }
}

// Decode, a CTA per chunk; offsets from k_tp_scan over the stream's size
// table.  A stream that does not fit its header, size table or levels sets
// HI_ECORRUPT and leaves those chunks' bytes unwritten.
__global__ void __launch_bounds__(kTpThreads, 4) k_tp_decode_chunks(const uint8_t* __restrict__ in, uint64_t in_len,
                                                                 uint64_t n, uint32_t nchunks,
                                                                 const uint64_t* __restrict__ offsets,
                                                                 uint8_t* __restrict__ out,
                                                                 uint32_t* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ uint32_t s_red[2 * (kTpThreads / 32)];
    int parity = 0;
    const uint32_t t = threadIdx.x;
    const bool hdr_ok = reinterpret_cast<const uint64_t*>(in)[0] == n &&
                        reinterpret_cast<const uint32_t*>(in)[2] == kTpChunk &&
                        reinterpret_cast<const uint32_t*>(in)[3] == nchunks;
    if (!hdr_ok) {
        if (blockIdx.x == 0 && t == 0) set_status(status, HI_ECORRUPT);
        return;
    }
    uint8_t* pay = tsm + kTpLevelBytes;
    const uint64_t hb = tp_header_bytes(nchunks);
    const bool vec_out = (reinterpret_cast<uintptr_t>(out) & 7u) == 0;
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint32_t sz = reinterpret_cast<const uint32_t*>(in + 16)[k];
        const uint32_t pad = sz & ~kTpRaw;
        const bool raw = (sz & kTpRaw) != 0;
        const uint32_t m = (uint32_t)min((uint64_t)kTpChunk, n - (uint64_t)k * kTpChunk);
        const uint64_t off = offsets[k];
        bool ok = pad % 16 == 0 && off % 16 == 0 && pad <= (m + 15) / 16 * 16 && off >= hb && off + pad <= in_len;
        if (raw) ok = ok && pad >= m;
        uint8_t* o = out + (uint64_t)k * kTpChunk;
        if (!ok) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            continue;
        }
        const uint8_t* p = in + off;
        if (raw) {
            for (uint32_t i = t; i < m; i += blockDim.x) o[i] = p[i];
            continue;
        }
        for (uint32_t i = t; i < pad / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(pay)[i] = reinterpret_cast<const uint4*>(p)[i];
        const TpLevels T = tp_levels(m);
        if (T.L[T.R] > pad) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            __syncthreads();
            continue;
        }
        __syncthreads();
        uint8_t* top = tsm + tp_level_off(T.R);
        for (uint32_t i = t; i < T.L[T.R]; i += blockDim.x) top[i] = pay[i];
        __syncthreads();
        uint32_t q = T.L[T.R];
        bool good = true;
        for (int r = T.R - 1; r >= 0; --r) {
            uint8_t* v = tsm + tp_level_off(r);
            const uint32_t span = level_span(r), a = span * t;
            const uint64_t f = (a < T.L[r]) ? level_bits(tsm + tp_level_off(r + 1), r, t, T.L[r]) : 0ull;
            uint32_t c_tot;
            uint32_t rank = block_exscan((uint32_t)__popcll(f), s_red, parity, &c_tot);
            if (q + c_tot > pad) {
                good = false;
                break;
            }
            if (a < T.L[r]) {
                // v[a + i] = the kept byte of rank (set bits at or before a + i), 0 before the first
                for (uint32_t w0 = 0; w0 < span; w0 += 4) {
                    uint32_t word = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        rank += (uint32_t)((f >> (w0 + b)) & 1ull);
                        const uint32_t val = rank ? pay[q + rank - 1] : 0u;
                        word |= val << (8 * b);
                    }
                    reinterpret_cast<uint32_t*>(v + a)[w0 / 4] = word;
                }
            }
            q += c_tot;
            __syncthreads();
        }
        if (!good) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            __syncthreads();
            continue;
        }
        // bit planes back to bytes (the transpose is its own inverse), then TCMS1 back
        const uint8_t* u = tsm + tp_level_off(0);
        const uint32_t pl = T.L[0] / 8;
        if (64 * t < T.L[0]) {
            uint32_t qlo[8], qhi[8];
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) {
                const uint2 w = reinterpret_cast<const uint2*>(u + pp * pl)[t];
                qlo[pp] = w.x, qhi[pp] = w.y;
            }
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                // byte 7 - p of group g's transposed word = byte g of plane p's 8 bytes
                uint32_t h[8];
#pragma unroll
                for (int pp = 0; pp < 8; ++pp) h[7 - pp] = g < 4 ? qlo[pp] : qhi[pp];
                const uint32_t sel = (uint32_t)(g & 3) | ((uint32_t)(4 + (g & 3)) << 4);
                const uint32_t lo = __byte_perm(__byte_perm(h[0], h[1], sel), __byte_perm(h[2], h[3], sel), 0x5410);
                const uint32_t hi = __byte_perm(__byte_perm(h[4], h[5], sel), __byte_perm(h[6], h[7], sel), 0x5410);
                const uint64_t x = transpose8((uint64_t)lo | ((uint64_t)hi << 32));
                const uint32_t e0 = tcms1_inv_4((uint32_t)x), e1 = tcms1_inv_4((uint32_t)(x >> 32));
                const uint32_t e = 64 * t + 8 * g;
                if (vec_out && e + 8 <= m) {
                    reinterpret_cast<uint2*>(o + e)[0] = make_uint2(e0, e1);
                } else {
                    for (int b = 0; b < 8; ++b)
                        if (e + b < m) o[e + b] = (uint8_t)((b < 4 ? e0 : e1) >> (8 * (b & 3)));
                }
            }
        }
        __syncthreads();
    }
}

size_t tp_ws_bytes(uint64_t n)
{
    const uint64_t nc = (n + kTpChunk - 1) / kTpChunk;
    return (size_t)((4 * nc + 15) / 16 * 16 + 8 * nc + nc * kTpSlot + 16);
}

uint64_t tp_stream_bound(uint64_t n)
{
    const uint64_t nc = (n + kTpChunk - 1) / kTpChunk;
    return tp_header_bytes(nc) + nc * 16 + n + 15;
}

static int tp_grid(uint32_t nchunks, int num_sms)
{
    const uint32_t cap = (uint32_t)num_sms * 6;  // 6 CTAs of ~36 KB shared memory per SM
    return (int)(nchunks < cap ? (nchunks ? nchunks : 1) : cap);
}

cudaError_t launch_tp_encode(const uint8_t* in, uint64_t n, uint8_t* out, uint64_t* len, void* ws, int num_sms,
                             cudaStream_t st)
{
    const uint32_t nc = (uint32_t)((n + kTpChunk - 1) / kTpChunk);
    uint8_t* w = static_cast<uint8_t*>(ws);
    uint32_t* sizes = reinterpret_cast<uint32_t*>(w);
    uint64_t* offsets = reinterpret_cast<uint64_t*>(w + (4 * (uint64_t)nc + 15) / 16 * 16);
    uint8_t* slots = reinterpret_cast<uint8_t*>(offsets + nc);
    slots = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(slots) + 15) & ~(uintptr_t)15);
    if (nc) {
        k_tp_encode_chunks<<<tp_grid(nc, num_sms), kTpThreads, kTpLevelBytes + kTpChunk, st>>>(in, n, slots, sizes,
                                                                                              nc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_tp_scan<<<1, 1024, 0, st>>>(sizes, nc, n, offsets, out, len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !nc) return e;
    k_tp_gather<<<tp_grid(nc, num_sms), 256, 0, st>>>(slots, sizes, offsets, nc, out);
    return cudaGetLastError();
}

cudaError_t launch_tp_decode(const uint8_t* in, uint64_t in_len, uint64_t n, uint8_t* out, uint32_t* status, void* ws,
                             int num_sms, cudaStream_t st)
{
    const uint32_t nc = (uint32_t)((n + kTpChunk - 1) / kTpChunk);
    if (!nc) return cudaSuccess;
    uint64_t* offsets = static_cast<uint64_t*>(ws);
    k_tp_scan<<<1, 1024, 0, st>>>(reinterpret_cast<const uint32_t*>(in + 16), nc, n, offsets, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tp_decode_chunks<<<tp_grid(nc, num_sms), kTpThreads, kTpLevelBytes + kTpChunk, st>>>(in, in_len, n, nc, offsets,
                                                                                          out, status);
    return cudaGetLastError();
}

}  // namespace hi
