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
// A CTA per chunk.  Thread t of the T = m' / 64 active threads holds
// elements 64 t .. 64 t + 63 as their bit-plane pieces in registers: bytes
// 8 t .. 8 t + 7 of each plane p, i.e. level-0 positions p m'/8 + 8 t ..,
// whose bitmap byte is byte p T + t of level 1.  TCMS1 is applied in the
// plane domain: with B_p the planes of the bytes themselves, the planes of
// TCMS1(b) are B_{p+1} ^ B_0 (p < 7) and B_0 (p = 7).  Levels 1 and 2 (at
// most 2048 and 256 bytes) are the work of warp 0.  The block needs one
// prefix sum per chunk: the kept counts of the 8 planes, four packed words
// per thread.  Encoding: kept bytes compacted with byte permutes from a
// 256-entry selector table into the payload staged in shared memory, then a
// scratch slot per chunk; a scan of the sizes; a gather of the payloads.
// Decoding: the scan, then per chunk the levels top down, each piece's 8
// values picked with byte permutes from the kept bytes (value i = the kept
// byte of rank popcount(bitmap[0..i]) - 1), and the planes back to bytes.
#include "hi_internal.h"
#include "hi_device.cuh"

namespace hi {

constexpr uint32_t kTpChunk = 16384;
constexpr uint32_t kTpRaw = 0x80000000u;
constexpr uint32_t kTpSlot = kTpChunk + 64;  // scratch bytes per chunk (16-byte multiple)
constexpr int kTpThreads = 256;
constexpr int kTpBlocksPerSm = 4;
constexpr int kTpMaxLevels = 6;
static_assert(kTpThreads == 256 && kTpChunk == 16384, "a thread per 64 elements, warp 0 covers levels 1 and 2");

__host__ __device__ constexpr uint64_t tp_header_bytes(uint64_t nchunks) { return (16 + 4 * nchunks + 15) / 16 * 16; }

struct TpLevels {
    uint32_t L[kTpMaxLevels];
    int R;  // top level (at most 3 for m <= 16384)
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

// Bit i of the result set when byte i of the piece (lo, hi) differs from the
// byte before it; pv = the byte before the piece.
__device__ __forceinline__ uint32_t piece_flags(uint32_t lo, uint32_t hi, uint32_t pv)
{
    return diff_flags4(lo, pv << 24) | (diff_flags4(hi, lo) << 4);
}

// The bit planes of 64 bytes e[0..15] (little-endian words): P[2p], P[2p+1]
// = the 8 bytes of plane p (bit 7 - p of each byte), element 8 j + b at bit
// b of byte j.
__device__ __forceinline__ void tp_planes(const uint32_t e[16], uint32_t P[16])
{
    uint64_t tr[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) tr[g] = transpose8((uint64_t)e[2 * g] | ((uint64_t)e[2 * g + 1] << 32));
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int b = 7 - p;  // byte of each transposed group holding plane p
        uint32_t h[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) h[g] = (uint32_t)(tr[g] >> (b >= 4 ? 32 : 0));
        const uint32_t sel = (uint32_t)(b & 3) | ((uint32_t)(4 + (b & 3)) << 4);
        P[2 * p] = __byte_perm(__byte_perm(h[0], h[1], sel), __byte_perm(h[2], h[3], sel), 0x5410);
        P[2 * p + 1] = __byte_perm(__byte_perm(h[4], h[5], sel), __byte_perm(h[6], h[7], sel), 0x5410);
    }
}

// The inverse of tp_planes (the transpose is its own inverse).
__device__ __forceinline__ void tp_unplanes(const uint32_t P[16], uint32_t e[16])
{
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        // byte 7 - p of group g's transposed word = byte g of plane p's 8 bytes
        uint32_t h[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) h[7 - p] = g < 4 ? P[2 * p] : P[2 * p + 1];
        const uint32_t sel = (uint32_t)(g & 3) | ((uint32_t)(4 + (g & 3)) << 4);
        const uint32_t lo = __byte_perm(__byte_perm(h[0], h[1], sel), __byte_perm(h[2], h[3], sel), 0x5410);
        const uint32_t hi = __byte_perm(__byte_perm(h[4], h[5], sel), __byte_perm(h[6], h[7], sel), 0x5410);
        const uint64_t x = transpose8((uint64_t)lo | ((uint64_t)hi << 32));
        e[2 * g] = (uint32_t)x;
        e[2 * g + 1] = (uint32_t)(x >> 32);
    }
}

// TCMS1 in the plane domain and back: bit j of (b << 1) ^ (b >> 7) is bit
// j - 1 of b xor its sign (j > 0) and the sign (j = 0).
__device__ __forceinline__ void tp_tcms_planes(uint32_t P[16])
{
    const uint32_t s0 = P[0], s1 = P[1];
#pragma unroll
    for (int p = 0; p < 7; ++p) {
        P[2 * p] = P[2 * p + 2] ^ s0;
        P[2 * p + 1] = P[2 * p + 3] ^ s1;
    }
    P[14] = s0;
    P[15] = s1;
}
__device__ __forceinline__ void tp_tcms_planes_inv(uint32_t P[16])
{
    const uint32_t s0 = P[14], s1 = P[15];
#pragma unroll
    for (int p = 6; p >= 0; --p) {
        P[2 * p + 2] = P[2 * p] ^ s0;
        P[2 * p + 3] = P[2 * p + 1] ^ s1;
    }
    P[0] = s0;
    P[1] = s1;
}

__device__ __forceinline__ uint32_t warp_incl_sum(uint32_t c)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, c, d);
        if (lane >= (uint32_t)d) c += x;
    }
    return c;
}

// Exclusive prefix over the block of four words per thread (each word two
// 16-bit counts, added without carries between them) and the block's
// totals.  One barrier; part is written again only by the next call, which
// every thread reaches after its last read of this one.
__device__ __forceinline__ void block_scan4(const uint32_t W[4], uint32_t E[4], uint32_t Tt[4], uint4* part)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t I[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) I[j] = W[j];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, I[j], d);
            if (lane >= (uint32_t)d) I[j] += x;
        }
    }
    if (lane == 31) part[warp] = make_uint4(I[0], I[1], I[2], I[3]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) E[j] = I[j] - W[j], Tt[j] = 0u;
#pragma unroll
    for (uint32_t w = 0; w < kTpThreads / 32; ++w) {
        const uint4 v = part[w];
        const uint32_t b = w < warp ? 0xffffffffu : 0u;
        E[0] += v.x & b, E[1] += v.y & b, E[2] += v.z & b, E[3] += v.w & b;
        Tt[0] += v.x, Tt[1] += v.y, Tt[2] += v.z, Tt[3] += v.w;
    }
}

__device__ __forceinline__ uint32_t field16(const uint32_t W[4], int p) { return (W[p >> 1] >> (16 * (p & 1))) & 0xffffu; }

// The bytes of the piece (lo, hi) whose bits are set in f, in order, to
// dst[0 .. popc(f)): nibble j of lut[f] is the index of the j-th set bit.
__device__ __forceinline__ void tp_put(uint8_t* dst, uint32_t lo, uint32_t hi, uint32_t f, const uint32_t* lut)
{
    if (!f) return;
    const uint32_t sel = lut[f];
    const uint32_t a = __byte_perm(lo, hi, sel), b = __byte_perm(lo, hi, sel >> 16);
    const int c = __popc(f);
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (j < c) dst[j] = (uint8_t)((j < 4 ? a : b) >> (8 * (j & 3)));
}

// The 8 values of a piece with bitmap byte f, r0 set bits of its level
// before it, kept bytes at pay[q ..] (q >= 1): value i = the kept byte of
// rank r0 + popc(f & (2^(i+1) - 1)) - 1, 0 for rank -1.  Reads the words
// covering pay[q + r0 - 1 .. q + r0 + 8].
__device__ __forceinline__ uint2 tp_expand(const uint8_t* pay, uint32_t q, uint32_t r0, uint32_t f)
{
    const bool all = f == 0xffu;
    const uint32_t s = q + r0 - (all ? 0u : 1u);  // window start: the byte before the piece's first kept byte
    const uint32_t* w = reinterpret_cast<const uint32_t*>(pay + (s & ~3u));
    const uint32_t sh = 8u * (s & 3u);
    uint32_t lo = __funnelshift_r(w[0], w[1], sh);
    const uint32_t hi = __funnelshift_r(w[1], w[2], sh);
    uint32_t sel = 0x76543210u;
    if (!all) {
        if (r0 == 0) lo &= 0xffffff00u;  // no kept byte before: the value 0
        // nibble i = popc(f & (2^(i+1) - 1)) <= 7: the bits spread to nibbles, prefix-summed by a multiply
        uint32_t x = f;
        x = (x | (x << 12)) & 0x000f000fu;
        x = (x | (x << 6)) & 0x03030303u;
        x = (x | (x << 3)) & 0x11111111u;
        sel = x * 0x11111111u;
    }
    return make_uint2(__byte_perm(lo, hi, sel), __byte_perm(lo, hi, sel >> 16));
}

struct TpEncSmem {
    alignas(16) uint8_t pay[kTpChunk + 16];     // the payload
    alignas(16) uint8_t b1[kTpChunk / 8 + 16];  // level 1 (the bitmap of level 0)
    alignas(16) uint8_t b2[kTpChunk / 64 + 16];
    alignas(16) uint8_t b3[kTpChunk / 512 + 16];
    uint4 part[kTpThreads / 32];
    uint2 last[kTpThreads];  // the last byte of each plane piece (lane 31 and thread T - 1)
    uint32_t lut[256];
    uint32_t tot12;          // kept counts of levels 1 (low half) and 2
};

__global__ void __launch_bounds__(kTpThreads, kTpBlocksPerSm) k_tp_encode_chunks(const uint8_t* __restrict__ in,
                                                                                 uint64_t n,
                                                                                 uint8_t* __restrict__ slots,
                                                                                 uint32_t* __restrict__ sizes,
                                                                                 uint32_t nchunks)
{
    __shared__ TpEncSmem S;
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    {
        uint32_t sel = 0, j = 0;
        for (int i = 0; i < 8; ++i)
            if ((t >> i) & 1u) sel |= (uint32_t)i << (4 * j++);
        S.lut[t] = sel;  // read after the first chunk's barriers
    }
    const bool al16 = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint8_t* s = in + (uint64_t)k * kTpChunk;
        const uint32_t m = (uint32_t)min((uint64_t)kTpChunk, n - (uint64_t)k * kTpChunk);
        const TpLevels L = tp_levels(m);
        const uint32_t T = L.L[0] / 64;
        const bool act = t < T;
        uint32_t P[16];
        {
            uint32_t e[16];
            if (act && al16 && 64 * t + 64 <= m) {
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4*>(s + 64 * t) + g);
                    e[4 * g] = v.x, e[4 * g + 1] = v.y, e[4 * g + 2] = v.z, e[4 * g + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int w = 0; w < 16; ++w) {
                    uint32_t x = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t i = 64 * t + 4 * w + b;
                        if (act && i < m) x |= (uint32_t)s[i] << (8 * b);  // zero padding past m
                    }
                    e[w] = x;
                }
            }
            tp_planes(e, P);
            tp_tcms_planes(P);
        }
        if (act && (lane == 31u || t == T - 1)) {
            const uint32_t lo4 = __byte_perm(__byte_perm(P[1], P[3], 0x73), __byte_perm(P[5], P[7], 0x73), 0x5410);
            const uint32_t hi4 = __byte_perm(__byte_perm(P[9], P[11], 0x73), __byte_perm(P[13], P[15], 0x73), 0x5410);
            S.last[t] = make_uint2(lo4, hi4);
        }
        __syncthreads();  // 1: the edge bytes
        // level-0 flags: the byte before a piece is in the previous lane's piece, or
        // (lane 0) the previous warp's last, or (t = 0) the end of the previous plane
        uint2 lw = make_uint2(0u, 0u);
        if (lane == 0 && act) {
            if (t) {
                lw = S.last[t - 1];
            } else {
                const uint2 z = S.last[T - 1];
                lw = make_uint2(z.x << 8, __funnelshift_l(z.x, z.y, 8));
            }
        }
        uint32_t fw[2] = {0u, 0u}, W[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const uint32_t up = __shfl_up_sync(0xffffffffu, P[2 * p + 1], 1);
            const uint32_t pv = lane ? (up >> 24) : (((p < 4 ? lw.x : lw.y) >> (8 * (p & 3))) & 0xffu);
            const uint32_t f = act ? piece_flags(P[2 * p], P[2 * p + 1], pv) : 0u;
            if (act) S.b1[p * T + t] = (uint8_t)f;
            fw[p >> 2] |= f << (8 * (p & 3));
            W[p >> 1] |= (uint32_t)__popc(f) << (16 * (p & 1));
        }
        uint32_t E[4], Tt[4];
        block_scan4(W, E, Tt, S.part);  // 2: level 1 complete
        uint32_t tot0 = 0;
#pragma unroll
        for (int p = 0; p < 8; ++p) tot0 += field16(Tt, p);
        const uint32_t top = L.L[L.R];
        if (warp == 0) {
            // levels 1 (64 positions a lane) and 2 (8 a lane) with their bitmaps
            uint64_t f1 = 0;
            uint32_t f2 = 0;
            if (L.R >= 2 && 64 * lane < L.L[1]) {
                f1 = range_flags<16>(S.b1, 64 * lane, L.L[1]);
                reinterpret_cast<uint2*>(S.b2)[lane] = make_uint2((uint32_t)f1, (uint32_t)(f1 >> 32));
            }
            __syncwarp();
            if (L.R >= 3 && 8 * lane < L.L[2]) {
                f2 = (uint32_t)range_flags<2>(S.b2, 8 * lane, L.L[2]);
                S.b3[lane] = (uint8_t)f2;
            }
            __syncwarp();
            const uint32_t c = (uint32_t)__popcll(f1) | ((uint32_t)__popc(f2) << 16);
            const uint32_t incl = warp_incl_sum(c);
            const uint32_t tot12 = __shfl_sync(0xffffffffu, incl, 31), ex = incl - c;
            const uint32_t base2 = top, base1 = top + (tot12 >> 16), base0 = base1 + (tot12 & 0xffffu);
            if (L.R >= 1 && base0 + tot0 <= m) {
                const uint8_t* tb = L.R == 1 ? S.b1 : (L.R == 2 ? S.b2 : S.b3);
                for (uint32_t i = lane; i < top; i += 32) S.pay[i] = tb[i];
                if (f2) {
                    const uint2 v = reinterpret_cast<const uint2*>(S.b2)[lane];
                    tp_put(S.pay + base2 + (ex >> 16), v.x, v.y, f2, S.lut);
                }
                uint32_t pos = base1 + (ex & 0xffffu);
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const uint32_t fg = (uint32_t)(f1 >> (8 * g)) & 0xffu;
                    const uint2 v = reinterpret_cast<const uint2*>(S.b1 + 64 * lane)[g];
                    tp_put(S.pay + pos, v.x, v.y, fg, S.lut);
                    pos += (uint32_t)__popc(fg);
                }
            }
            if (lane == 0) S.tot12 = tot12;
        }
        __syncthreads();  // 3: levels 1, 2 and their kept bytes placed
        const uint32_t tot12 = S.tot12;
        const uint32_t base0 = top + (tot12 >> 16) + (tot12 & 0xffffu);
        const uint32_t total = L.R ? base0 + tot0 : top;
        const bool raw = total > m;
        if (!raw && act) {
            if (L.R == 0) {  // m' = 64: level 0 is the top, stored as is
#pragma unroll
                for (int p = 0; p < 8; ++p)
                    reinterpret_cast<uint2*>(S.pay)[p] = make_uint2(P[2 * p], P[2 * p + 1]);
            } else {
                uint32_t pb = base0;
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    tp_put(S.pay + pb + field16(E, p), P[2 * p], P[2 * p + 1], (fw[p >> 2] >> (8 * (p & 3))) & 0xffu,
                           S.lut);
                    pb += field16(Tt, p);
                }
            }
        }
        __syncthreads();  // 4: the payload
        uint8_t* slot = slots + (uint64_t)k * kTpSlot;
        const uint32_t len = raw ? m : total;
        const uint32_t pad = (len + 15) / 16 * 16;
        for (uint32_t i = t; i < pad / 16; i += blockDim.x) {
            uint32_t w[4];
            if (!raw) {
                const uint4 v = reinterpret_cast<const uint4*>(S.pay)[i];
                w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
            } else if (al16 && 16 * i + 16 <= m) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(s) + i);
                w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
            } else {
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    if (!(b & 3)) w[b >> 2] = 0u;
                    if (16 * i + b < m) w[b >> 2] |= (uint32_t)s[16 * i + b] << (8 * (b & 3));
                }
            }
            if (16 * i + 16 > len) {  // zero past the end
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int keep = (int)len - (int)(16 * i + 4 * b);
                    w[b] &= keep >= 4 ? 0xffffffffu : (keep <= 0 ? 0u : (1u << (8 * keep)) - 1u);
                }
            }
            reinterpret_cast<uint4*>(slot)[i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (t == 0) sizes[k] = pad | (raw ? kTpRaw : 0u);
    }
}

// Exclusive scan of the padded sizes (one CTA): offsets[k] = header +
// sum of sizes before k; with out != nullptr also writes the stream header
// and size table, and the stream length to *len.  A thread takes
// kTpScanPer consecutive entries (16-byte loads and stores where whole),
// one block scan of the per-thread sums for every 1024 kTpScanPer entries.
// sizes, offsets and out are 16-byte aligned.
constexpr uint32_t kTpScanPer = 16;

__global__ void __launch_bounds__(1024) k_tp_scan(const uint32_t* __restrict__ sizes, uint32_t nchunks, uint64_t n,
                                                  uint64_t* __restrict__ offsets, uint8_t* __restrict__ out,
                                                  uint64_t* __restrict__ len)
{
    __shared__ uint64_t s_part[32];
    __shared__ uint64_t s_base;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = tp_header_bytes(nchunks);
    __syncthreads();
    uint32_t* table = out ? reinterpret_cast<uint32_t*>(out + 16) : nullptr;
    for (uint32_t c0 = 0; c0 < nchunks; c0 += blockDim.x * kTpScanPer) {
        const uint32_t k0 = c0 + threadIdx.x * kTpScanPer;
        const bool whole = k0 + kTpScanPer <= nchunks;
        uint32_t v[kTpScanPer];
        if (whole) {
#pragma unroll
            for (uint32_t j = 0; j < kTpScanPer / 4; ++j) {
                const uint4 q = reinterpret_cast<const uint4*>(sizes + k0)[j];
                v[4 * j] = q.x, v[4 * j + 1] = q.y, v[4 * j + 2] = q.z, v[4 * j + 3] = q.w;
            }
        } else {
#pragma unroll
            for (uint32_t j = 0; j < kTpScanPer; ++j) v[j] = k0 + j < nchunks ? sizes[k0 + j] : 0u;
        }
        uint64_t sum = 0;
#pragma unroll
        for (uint32_t j = 0; j < kTpScanPer; ++j) sum += v[j] & ~kTpRaw;
        uint64_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += t;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        uint64_t o = s_base + incl - sum;
        for (uint32_t w = 0; w < warp; ++w) o += s_part[w];
        if (whole) {
#pragma unroll
            for (uint32_t j = 0; j < kTpScanPer; j += 2) {
                const uint64_t a = o;
                o += v[j] & ~kTpRaw;
                reinterpret_cast<ulonglong2*>(offsets + k0)[j / 2] = make_ulonglong2(a, o);
                o += v[j + 1] & ~kTpRaw;
            }
            if (table) {
#pragma unroll
                for (uint32_t j = 0; j < kTpScanPer / 4; ++j)
                    reinterpret_cast<uint4*>(table + k0)[j] = make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
        } else {
#pragma unroll
            for (uint32_t j = 0; j < kTpScanPer; ++j) {
                if (k0 + j < nchunks) {
                    offsets[k0 + j] = o;
                    if (table) table[k0 + j] = v[j];
                }
                o += v[j] & ~kTpRaw;
            }
        }
        __syncthreads();  // s_part read; the last thread's running sum is the round's end
        if (threadIdx.x == blockDim.x - 1) s_base = o;
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
// HI_ECORRUPT and leaves those chunks' bytes unwritten.  Two payload
// buffers, alternating per loaded payload: the barrier after a load
// separates the load of the next-but-one from the last reads of a buffer.
struct TpDecSmem {
    alignas(16) uint8_t pay[2][kTpChunk + 16];
    alignas(16) uint8_t v1[kTpChunk / 8 + 16];  // level 1
    alignas(16) uint8_t v2[kTpChunk / 64 + 16];
    uint4 part[kTpThreads / 32];
    uint32_t q0, good;  // start of level 0's kept bytes; levels above consistent
};

__global__ void __launch_bounds__(kTpThreads, kTpBlocksPerSm) k_tp_decode_chunks(
    const uint8_t* __restrict__ in, uint64_t in_len, uint64_t n, uint32_t nchunks,
    const uint64_t* __restrict__ offsets, uint8_t* __restrict__ out, uint32_t* __restrict__ status)
{
    __shared__ TpDecSmem S;
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const bool hdr_ok = reinterpret_cast<const uint64_t*>(in)[0] == n &&
                        reinterpret_cast<const uint32_t*>(in)[2] == kTpChunk &&
                        reinterpret_cast<const uint32_t*>(in)[3] == nchunks;
    if (!hdr_ok) {
        if (blockIdx.x == 0 && t == 0) set_status(status, HI_ECORRUPT);
        return;
    }
    const uint64_t hb = tp_header_bytes(nchunks);
    const bool vec_out = (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
    uint32_t it = 0;  // payloads loaded so far: each load is followed by a barrier before the next
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        uint8_t* pay = S.pay[it & 1u];
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
        ++it;
        const TpLevels L = tp_levels(m);
        if (L.L[L.R] > pad) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            __syncthreads();
            continue;
        }
        __syncthreads();  // 1: the payload
        if (warp == 0) {
            uint32_t q = L.L[L.R];
            bool good = true;
            if (L.R >= 3) {  // level 2; its bitmap is the top
                const uint32_t a = 8 * lane, Ln = L.L[2];
                uint32_t f = a < Ln ? (uint32_t)pay[lane] : 0u;
                if (a < Ln && a + 8 > Ln) f &= (1u << (Ln - a)) - 1u;
                const uint32_t c = (uint32_t)__popc(f), incl = warp_incl_sum(c);
                const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
                if (q + tot > pad) {
                    good = false;
                } else if (a < Ln) {
                    reinterpret_cast<uint2*>(S.v2)[lane] = tp_expand(pay, q, incl - c, f);
                }
                q += tot;
            }
            __syncwarp();
            if (L.R >= 2 && good) {  // level 1; its bitmap is level 2
                const uint8_t* bm = L.R >= 3 ? S.v2 : pay;
                const uint32_t a = 64 * lane, Ln = L.L[1];
                uint64_t f = 0;
                if (a < Ln) {
                    const uint2 b = reinterpret_cast<const uint2*>(bm)[lane];
                    f = (uint64_t)b.x | ((uint64_t)b.y << 32);
                    if (a + 64 > Ln) f &= (1ull << (Ln - a)) - 1ull;
                }
                const uint32_t c = (uint32_t)__popcll(f), incl = warp_incl_sum(c);
                const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
                if (q + tot > pad) {
                    good = false;
                } else if (a < Ln) {
                    uint32_t r = incl - c;
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const uint32_t fg = (uint32_t)(f >> (8 * g)) & 0xffu;
                        reinterpret_cast<uint2*>(S.v1 + a)[g] = tp_expand(pay, q, r, fg);
                        r += (uint32_t)__popc(fg);
                    }
                }
                q += tot;
            }
            if (lane == 0) S.q0 = q, S.good = good ? 1u : 0u;
        }
        __syncthreads();  // 2: levels 1 and 2
        const uint32_t q0 = S.q0;
        if (!S.good) {
            if (t == 0) set_status(status, HI_ECORRUPT);
            continue;
        }
        const uint32_t T = L.L[0] / 64;
        const bool act = t < T;
        uint32_t P[16];
        if (L.R == 0) {  // m' = 64: the top is level 0 (one active thread)
#pragma unroll
            for (int j = 0; j < 16; ++j) P[j] = act ? reinterpret_cast<const uint32_t*>(pay)[j] : 0u;
        } else {
            const uint8_t* bm = L.R == 1 ? pay : S.v1;
            uint32_t fw[2] = {0u, 0u}, W[4] = {0u, 0u, 0u, 0u};
            if (act) {
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const uint32_t f = bm[p * T + t];
                    fw[p >> 2] |= f << (8 * (p & 3));
                    W[p >> 1] |= (uint32_t)__popc(f) << (16 * (p & 1));
                }
            }
            uint32_t E[4], Tt[4];
            block_scan4(W, E, Tt, S.part);  // 3
            uint32_t tot0 = 0;
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) tot0 += field16(Tt, pp);
            if (q0 + tot0 > pad) {
                if (t == 0) set_status(status, HI_ECORRUPT);
                continue;
            }
            uint32_t pb = 0;
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) {
                const uint2 v = act ? tp_expand(pay, q0, pb + field16(E, pp), (fw[pp >> 2] >> (8 * (pp & 3))) & 0xffu)
                                    : make_uint2(0u, 0u);
                P[2 * pp] = v.x, P[2 * pp + 1] = v.y;
                pb += field16(Tt, pp);
            }
        }
        if (!act) continue;
        tp_tcms_planes_inv(P);
        uint32_t e[16];
        tp_unplanes(P, e);
        const uint32_t e0 = 64 * t;
        if (vec_out && e0 + 64 <= m) {
#pragma unroll
            for (int g = 0; g < 4; ++g)
                reinterpret_cast<uint4*>(o + e0)[g] = make_uint4(e[4 * g], e[4 * g + 1], e[4 * g + 2], e[4 * g + 3]);
        } else {
#pragma unroll
            for (int b = 0; b < 64; ++b)
                if (e0 + b < m) o[e0 + b] = (uint8_t)(e[b >> 2] >> (8 * (b & 3)));
        }
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
    const uint32_t cap = (uint32_t)num_sms * kTpBlocksPerSm;
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
        k_tp_encode_chunks<<<tp_grid(nc, num_sms), kTpThreads, 0, st>>>(in, n, slots, sizes,
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
    k_tp_decode_chunks<<<tp_grid(nc, num_sms), kTpThreads, 0, st>>>(in, in_len, n, nc, offsets,
                                                                                          out, status);
    return cudaGetLastError();
}

}  // namespace hi
